"""Saving and loading analysed plans (stc_plan_save / stc_plan_load), on the CPU.

A loaded plan must be the same plan: re-saving it gives the identical blob (the blob
holds every host array), every export and the plan info match the original, and the
task sets and supernodal layout it rebuilds on demand match.  Truncated, corrupted and
foreign blobs are refused.
"""
import numpy as np
import pytest

from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import build as B
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

EXPORTS = ["perm", "etree", "Lp", "Li", "tiles", "aind", "tasks", "value_map", "tile_offsets",
           "chunk_extents", "sn_nodes", "sn_rows", "sn_cells", "sn_tasks", "sn_dev_cells", "sn_dev_tasks",
           "sn_dev_upds", "sn_dev_maps", "sn_value_map", "sn_csc_map"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if B.stale():
        B.build()
    L.lib()


def _plans():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    yield "config1_nd", Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=64)
    Ap, Ai, Ax, coords = I.fem3d(10, 9, 8)
    yield "fem_dense_route", Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=32, route="dense", nd_leaf=32)
    Ap, Ai = I.band_pattern(3000, 70)
    yield "band_slices", Plan(3000, Ap, Ai, nb=64, ordering="natural", row_slices=4)
    Ap, Ai, _ = I.random_spd(700, 0.005, 2)
    yield "random_given", Plan(700, Ap, Ai, nb=24, perm=np.random.default_rng(1).permutation(700))
    Ap, Ai, Ax, coords = I.laplace2d_bordered(16, 16, 2)
    yield "supernodal_route", Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=32, route="supernodal")


PLANS = list(_plans())


@pytest.mark.parametrize("case", PLANS, ids=lambda c: c[0])
def test_round_trip_is_the_same_plan(case):
    _, P = case
    blob = P.save()
    Q = Plan.load(blob)
    assert Q.save() == blob
    assert Q.info == P.info
    for k in EXPORTS:
        assert np.array_equal(Q.export(k), P.export(k)), k
    assert Q.factor_bytes(3) == P.factor_bytes(3) and Q.workspace_bytes(5) == P.workspace_bytes(5)
    assert Q.route == P.route and Q.route_selected == P.route_selected


def test_refuses_truncated_corrupted_and_foreign_blobs():
    _, P = PLANS[0]
    blob = P.save()
    for bad in (blob[:10], blob[:-1], blob[:len(blob) // 2]):
        assert L.stc_plan_load(bad)[0] == L.STC_ERR_INVALID_PATTERN
    flipped = bytearray(blob)
    flipped[len(blob) // 3] ^= 0x40
    assert L.stc_plan_load(bytes(flipped))[0] == L.STC_ERR_INVALID_PATTERN
    foreign = bytearray(blob)
    foreign[0:8] = b"NOTAPLAN"
    assert L.stc_plan_load(bytes(foreign))[0] == L.STC_ERR_INVALID_PATTERN
    newer = bytearray(blob)
    newer[8] = 99  # format version
    assert L.stc_plan_load(bytes(newer))[0] == L.STC_ERR_UNSUPPORTED
    with pytest.raises(L.StcError):
        Plan.load(blob[:-8])


def test_save_size_query_and_short_buffer():
    _, P = PLANS[2]
    sz = L.C.c_size_t(0)
    assert L.lib().stc_plan_save(P.h, None, L.C.byref(sz)) == L.STC_OK
    assert sz.value == len(P.save())
    short = L.C.c_size_t(sz.value - 1)
    buf = L.C.create_string_buffer(sz.value)
    assert L.lib().stc_plan_save(P.h, buf, L.C.byref(short)) == L.STC_ERR_BUFFER_TOO_SMALL
    assert short.value == sz.value


def test_loaded_plan_survives_the_original():
    Ap, Ai = I.band_pattern(2000, 40)
    P = Plan(2000, Ap, Ai, nb=32, ordering="natural")
    ref = {k: P.export(k) for k in ("tiles", "value_map", "tasks")}
    blob = P.save()
    del P
    Q = Plan.load(blob)
    for k, v in ref.items():
        assert np.array_equal(Q.export(k), v)


def _fnv1a(b: bytes) -> int:
    h = 1469598103934665603
    for c in b:
        h = ((h ^ c) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _tiles_and_scalars(blob):
    """Byte offsets of the tile array and of two scalars in a saved blob (the format of
    plan_io.cpp: 32-byte header, scalars, then each array as a u64 count + elements)."""
    import struct
    so = L.C.sizeof(L.stc_options)
    sc = 32 + 32 + so + 12 + 32           # n..nnzA, options, 3 x int32, 4 doubles
    npartials_at, partial_off_at = sc + 16, sc + 24
    pos = 32 + 32 + so + 12 + 32 + 32 + 32 + 16
    perm_at = None
    for esize in (8, 8, 8, 4):            # perm, parent, Lp, Li
        (cnt,) = struct.unpack_from("<Q", blob, pos)
        if perm_at is None:
            perm_at = pos + 8
        pos += 8 + cnt * esize
    (ntiles,) = struct.unpack_from("<Q", blob, pos)
    return pos + 8, ntiles, npartials_at, partial_off_at, perm_at


def test_refuses_intact_but_inconsistent_blobs():
    # a blob with a valid checksum whose contents disagree with the plan's dimensions
    # (an edited blob, or one written by a build with another layout) must never reach
    # a kernel: each edit below is re-checksummed and must still be refused
    import struct
    Ap, Ai, _ = I.tridiag(300, 0)
    P = Plan(300, Ap, Ai, nb=32, ordering="natural", route="semisparse")
    blob = P.save()
    tiles_at, ntiles, np_at, po_at, perm_at = _tiles_and_scalars(blob)
    assert ntiles == P.info["ntiles"]
    (npartials,) = struct.unpack_from("<q", blob, np_at)
    (partial_off,) = struct.unpack_from("<q", blob, po_at)
    assert npartials == P.info["nt"]
    T = P.export("tiles")
    off_tile = int(np.nonzero(T[:, 0] != T[:, 1])[0][-1])
    diag_tile = int(np.nonzero(T[:, 0] == T[:, 1])[0][-1])

    def resign(b):
        b = bytearray(b)
        b[24:32] = struct.pack("<Q", _fnv1a(bytes(b[32:])))
        return bytes(b)

    assert Plan.load(resign(blob)).save() == blob  # re-signing alone changes nothing

    def edited(tile, field_at, fmt, value):
        b = bytearray(blob)
        struct.pack_into(fmt, b, tiles_at + 56 * tile + field_at, value)
        return resign(b)

    bad = {
        "footprint past the tile area": edited(off_tile, 0, "<q", partial_off - 1),
        "negative offset": edited(off_tile, 0, "<q", -8),
        "unknown tile kind": edited(diag_tile, 16, "<i", 7),
        "logdet slot out of range": edited(diag_tile, 48, "<i", npartials),
        "band wider than the tile": edited(diag_tile, 32, "<i", 32),
        "stored width past the tile": edited(off_tile, 20, "<i", 33),
    }
    b = bytearray(blob)
    b[perm_at:perm_at + 8] = b[perm_at + 8:perm_at + 16]   # perm[0] = perm[1]
    bad["perm not a permutation"] = resign(b)
    for what, blob2 in bad.items():
        assert L.stc_plan_load(blob2)[0] == L.STC_ERR_INVALID_PATTERN, what
