"""Host analysis (libstc.so, no GPU needed) against the oracle and the paper's examples."""
import json
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import build as B
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if B.stale():
        B.build()
    L.lib()


def test_library_exports_every_header_symbol():
    hdr = open(os.path.join(ROOT, "include", "stc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = sorted(set(re.findall(r"\b(stc_[a-z_0-9]+)\s*\(", hdr)))
    assert declared, "no declarations found"
    lib = L.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTED) == declared


def test_binding_refuses_pageable_host_inputs():
    # inputs the kernels read may be device tensors or pinned host tensors (read in place);
    # pageable host memory is refused before any call, outputs must be device tensors
    torch = pytest.importorskip("torch")
    x = torch.zeros(3, dtype=torch.float64)
    with pytest.raises(ValueError):
        L._in_ptr(x)
    with pytest.raises(ValueError):
        L._dev_ptr(x)


def _cases():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    yield "c1_nd_nb64", len(Ap) - 1, Ap, Ai, coords, dict(nb=64, ordering="nd"), None
    Ap, Ai = I.band_pattern(5000, 200)
    yield "band_nb128", 5000, Ap, Ai, None, dict(nb=128, ordering="natural"), None
    Ap, Ai, coords = I.stcov_pattern(12, 10, 6, 4)
    yield "stcov_small_nd_nb32", len(Ap) - 1, Ap, Ai, coords, dict(nb=32, ordering="nd"), None
    Ap, Ai, Ax, coords = I.fem3d(9, 8, 7)
    yield "fem3d_nd_nb16", len(Ap) - 1, Ap, Ai, coords, dict(nb=16, ordering="nd", nd_leaf=20), None
    for seed, (n, d) in enumerate([(300, 0.01), (257, 0.03), (64, 0.2)]):
        Ap, Ai, _ = I.random_spd(n, d, seed)
        perm = np.random.default_rng(seed + 5).permutation(n)
        yield "random%d_given" % seed, n, Ap, Ai, None, dict(nb=8 * (seed + 1)), perm


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_symbolic_bit_exact_vs_oracle(case):
    name, n, Ap, Ai, coords, kw, perm = case
    P = Plan(n, Ap, Ai, coords=coords, perm=perm, route="semisparse", **kw)
    if kw.get("ordering") == "nd":
        operm = O.nd_lattice(coords, kw.get("nd_leaf", 64))
    elif perm is not None:
        operm = perm
    else:
        operm = np.arange(n)
    assert np.array_equal(P.export("perm"), operm)
    F = O.OracleFactor(n, Ap, Ai, operm)
    assert np.array_equal(P.export("etree"), F.parent)
    assert np.array_equal(P.export("Lp"), F.Lp)
    assert np.array_equal(P.export("Li"), F.Li)
    t = F.tile_map(kw["nb"])
    T = P.export("tiles")
    ref = np.stack([t["I"], t["J"], t["nact"], t["aoff"], t["contig"], t["full"], t["kd"],
                    t["r0"], t["r1"]], axis=1)
    assert np.array_equal(T, ref)
    assert np.array_equal(P.export("aind"), t["aind"])
    assert np.array_equal(P.export("tasks"), t["tasks"])
    f = F.features(kw["nb"], t)
    assert P.info["phi"] == pytest.approx(f["phi"], rel=1e-12)
    assert P.info["rho"] == pytest.approx(f["rho"], rel=1e-12)
    assert P.info["sigma"] == pytest.approx(f["sigma"], rel=1e-12)
    assert P.info["route_selected"] == O.select_route(**f)
    assert P.info["nnzL"] == F.nnzL


def test_paper_banded_tile_layout():
    """Sec. 4.3 worked example: a_ij (i<=j) of the kd=2 tile sits at (kd+i-j, j)."""
    g = json.load(open(os.path.join(GOLD, "paper_banded_diag_tile.json")))
    m, kd = g["nb"], g["kd"]
    A = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            if abs(i - j) <= kd:
                A[i, j] = 4.0 if i == j else -0.5
    Ap, Ai, _ = I.lower_csc(sp.csc_matrix(A))
    P = Plan(m, Ap, Ai, nb=8, route="semisparse", ordering="natural")
    vm = P.export("value_map")
    off0 = P.export("tile_offsets")[0]
    col = np.repeat(np.arange(m), np.diff(Ap))
    for e in range(len(Ai)):
        r, c = Ai[e], col[e]          # L entry (r, c) = (L^T) entry (i=c, j=r)
        pos = int(vm[e] - off0)
        q, j = pos % (kd + 1), pos // (kd + 1)
        assert g["packed"][q][j] == "a%d%d" % (c, r)


def test_paper_active_column_storage():
    """Sec. 4.1 worked example: stored n_b x |A| buffer, stored column j' = aind index."""
    g = json.load(open(os.path.join(GOLD, "paper_active_column_tile.json")))
    nb = 8
    n = 2 * nb
    A = np.eye(n) * 10.0
    for r, c in g["entries_row_col"]:
        A[nb + r, c] = A[c, nb + r] = 0.5
    Ap, Ai, _ = I.lower_csc(sp.csc_matrix(A))
    P = Plan(n, Ap, Ai, nb=nb, route="semisparse", ordering="natural")
    T = P.export("tiles")
    k = int(np.nonzero((T[:, 0] == 1) & (T[:, 1] == 0))[0][0])
    aind = P.export("aind")[T[k, 3]:T[k, 3] + T[k, 2]]
    assert aind.tolist() == g["aind"]
    offs = P.export("tile_offsets")
    vm = P.export("value_map")
    col = np.repeat(np.arange(n), np.diff(Ap))
    for e in range(len(Ai)):
        if Ai[e] >= nb and col[e] < nb:
            r, c = Ai[e] - nb, col[e]
            assert vm[e] == offs[k] + r + g["aind"].index(c) * nb
    # the tile occupies n_b x |A| doubles: the next tile starts 3 columns later (32B aligned)
    assert offs[k + 1] - offs[k] == nb * len(g["aind"])


def test_dense_route_stores_full_tiles():
    Ap, Ai, Ax, coords = I.laplace2d_bordered(12, 12, 2)
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=16, route="dense")
    assert P.route == "dense"
    offs = P.export("tile_offsets")
    assert np.all(np.diff(offs) == 16 * 16)
    assert P.info["stored_entries"] == 16 * 16 * P.info["ntiles"]


def test_value_map_is_injective_and_inside_factor():
    Ap, Ai, _ = I.random_spd(200, 0.02, 3)
    P = Plan(200, Ap, Ai, nb=16, ordering="rcm", route="semisparse")
    vm = P.export("value_map")
    assert len(np.unique(vm)) == len(vm)
    assert vm.min() >= 0 and vm.max() < P.info["factor_doubles"]


def test_rcm_recovers_band():
    n, bw = 400, 3
    Ap, Ai = I.band_pattern(n, bw)
    p = np.random.default_rng(0).permutation(n)
    A = sp.csc_matrix((np.ones(len(Ai)), Ai, Ap), shape=(n, n))
    A = (A + A.T)[p][:, p]
    Bp, Bi, _ = I.lower_csc(A)
    P = Plan(n, Bp, Bi, nb=16, ordering="rcm")
    perm = P.export("perm")
    assert np.array_equal(np.sort(perm), np.arange(n))
    Q = A[perm][:, perm].tocoo()
    assert np.max(np.abs(Q.row - Q.col)) <= 2 * bw


def test_auto_ordering_keeps_natural_for_band():
    Ap, Ai = I.band_pattern(2000, 50)
    P = Plan(2000, Ap, Ai, nb=64)
    assert P.info["ordering"] == L.STC_ORDER_NATURAL
    assert P.info["phi"] == 1.0
    assert P.route == "semisparse"


def test_c2_band_structure_and_flops():
    n, bw, nb = 200_000, 200, 128
    Ap, Ai = I.band_pattern(n, bw)
    P = Plan(n, Ap, Ai, nb=nb, ordering="natural", route="semisparse")
    i = P.info
    assert i["nt"] == 1563 and i["phi"] == 1.0
    assert i["nnzL"] == len(Ai)
    cc = np.diff(Ap).astype(float)
    assert i["flops_alg"] == pytest.approx(np.sum(cc * cc))
    T = P.export("tiles")
    diag = T[:, 0] == T[:, 1]
    assert np.all(T[diag][:-1, 6] == nb - 1)
    far = T[:, 0] == T[:, 1] + 2
    assert np.all(T[far][:, 2] == 72) and np.all(T[far][:, 4] == 1)


@pytest.mark.parametrize("bad", ["unsorted", "nodiag", "upper", "outofrange"])
def test_invalid_patterns_rejected(bad):
    Ap, Ai, _ = I.tridiag(10, 0)
    Ai = Ai.copy(); Ap = Ap.copy()
    if bad == "unsorted":
        Ai[Ap[3]:Ap[4]] = Ai[Ap[3]:Ap[4]][::-1]
    elif bad == "nodiag":
        Ai[Ap[5]] = 7
    elif bad == "upper":
        Ai[Ap[4] + 1] = 2
    else:
        Ai[Ap[8] + 1] = 10
    rc, h = L.stc_analyze(10, Ap, Ai)
    assert rc == L.STC_ERR_INVALID_PATTERN and not h.value


def test_unsupported_options_rejected():
    Ap, Ai, _ = I.tridiag(10, 0)
    o = L.stc_options_default()
    o.nb = 100
    assert L.stc_analyze(10, Ap, Ai, None, o)[0] == L.STC_ERR_UNSUPPORTED
    o = L.stc_options_default()
    o.ordering = L.STC_ORDER_ND
    coords = np.full((10, 3), 0.5)
    assert L.stc_analyze(10, Ap, Ai, coords, o)[0] == L.STC_ERR_UNSUPPORTED
    o = L.stc_options_default()
    o.row_slices = 3
    assert L.stc_analyze(10, Ap, Ai, None, o)[0] == L.STC_ERR_INVALID_ARG
    o = L.stc_options_default()
    o.replay_ctas = -1
    assert L.stc_analyze(10, Ap, Ai, None, o)[0] == L.STC_ERR_INVALID_ARG


def test_export_buffer_too_small():
    Ap, Ai, _ = I.tridiag(10, 0)
    P = Plan(10, Ap, Ai, nb=8)
    sz = L.C.c_size_t(8)
    buf = np.empty(1, dtype=np.int64)
    rc = L.lib().stc_plan_export(P.h, L.STC_EXPORT_PERM, buf.ctypes.data_as(L.C.c_void_p), L.C.byref(sz))
    assert rc == L.STC_ERR_BUFFER_TOO_SMALL and sz.value == 80


def _chunk_extents_brute(F, t, nb, n, dense):
    """Per off-diagonal tile and group of 16 stored columns, the structural row extent,
    from the oracle's symbolic structure of L."""
    out = np.full((len(t["I"]), 8, 2), -1, dtype=np.int64)
    for k, (I_, J_) in enumerate(zip(t["I"], t["J"])):
        if I_ == J_:
            continue
        if dense:
            cols = np.arange(nb)
        else:
            cols = t["aind"][t["aoff"][k]:t["aoff"][k] + t["nact"][k]]
        for q in range(0, len(cols), 16):
            lo, hi = nb, 0
            for lc in cols[q:q + 16]:
                j = J_ * nb + lc
                if j >= n:
                    continue
                rows = F.Li[F.Lp[j]:F.Lp[j + 1]]
                rows = rows[rows // nb == I_] - I_ * nb
                if len(rows):
                    lo, hi = min(lo, int(rows.min())), max(hi, int(rows.max()) + 1)
            out[k, q // 16] = (lo, hi)
    return out


@pytest.mark.parametrize("case", [c for c in _cases() if c[0] in ("c1_nd_nb64", "band_nb128",
                                                                  "stcov_small_nd_nb32", "random0_given",
                                                                  "random1_given")],
                         ids=lambda c: c[0])
@pytest.mark.parametrize("route", ["semisparse", "dense"])
def test_chunk_row_extents_vs_oracle_structure(case, route):
    name, n, Ap, Ai, coords, kw, perm = case
    P = Plan(n, Ap, Ai, coords=coords, perm=perm, route=route, **kw)
    F = O.OracleFactor(n, Ap, Ai, P.export("perm"))
    t = F.tile_map(kw["nb"])
    ext = P.export("chunk_extents")
    assert np.array_equal(ext, _chunk_extents_brute(F, t, kw["nb"], n, route == "dense"))


def test_strerror_names_every_code():
    codes = [L.STC_OK, L.STC_ERR_INVALID_ARG, L.STC_ERR_INVALID_PATTERN, L.STC_ERR_OUT_OF_MEMORY,
             L.STC_ERR_CUDA, L.STC_ERR_TIMEOUT, L.STC_ERR_UNSUPPORTED, L.STC_ERR_BUFFER_TOO_SMALL]
    names = [L.stc_strerror(c) for c in codes]
    assert len(set(names)) == len(codes) and all(names)
    assert L.stc_strerror(-99) == "unknown error" and L.stc_strerror(7) == "unknown error"
    with pytest.raises(L.StcError, match="invalid argument"):
        L.check(L.STC_ERR_INVALID_ARG, "here")


@pytest.mark.parametrize("seed", range(12))
def test_random_patterns_symbolic_and_extents_vs_oracle(seed):
    # random sizes, densities, tile sizes and orderings: every symbolic export and the
    # 16-column row extents against the oracle and brute force
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(20, 260))
    Ap, Ai, _ = I.random_spd(n, float(rng.uniform(0.005, 0.08)), seed)
    nb = int(rng.choice([8, 16, 24, 32, 64]))
    kind = ["natural", "rcm", "given"][seed % 3]
    perm = rng.permutation(n) if kind == "given" else None
    route = "dense" if seed % 4 == 0 else "semisparse"
    P = Plan(n, Ap, Ai, nb=nb, ordering=kind if perm is None else "auto", perm=perm, route=route)
    operm = P.export("perm")
    assert np.array_equal(np.sort(operm), np.arange(n))
    if perm is not None:
        assert np.array_equal(operm, perm)
    F = O.OracleFactor(n, Ap, Ai, operm)
    assert np.array_equal(P.export("etree"), F.parent)
    assert np.array_equal(P.export("Lp"), F.Lp)
    assert np.array_equal(P.export("Li"), F.Li)
    t = F.tile_map(nb)
    T = P.export("tiles")
    ref = np.stack([t["I"], t["J"], t["nact"], t["aoff"], t["contig"], t["full"], t["kd"],
                    t["r0"], t["r1"]], axis=1)
    assert np.array_equal(T, ref)
    assert np.array_equal(P.export("aind"), t["aind"])
    assert np.array_equal(P.export("tasks"), t["tasks"])
    assert np.array_equal(P.export("chunk_extents"), _chunk_extents_brute(F, t, nb, n, route == "dense"))


def _plan_exports(P):
    names = ["perm", "etree", "Lp", "Li", "tiles", "aind", "tasks", "value_map", "tile_offsets",
             "chunk_extents"]
    return {k: P.export(k) for k in names}


@pytest.mark.parametrize("case", ["fem", "band", "random"])
def test_plan_independent_of_host_threads(case):
    # the analysis runs its symbolic factorization, tile map and maps on several host
    # threads; every output must be the same for any thread count
    if case == "fem":
        Ap, Ai, Ax, coords = I.fem3d(16, 16, 16)
        kw = dict(coords=coords, nb=32, route="dense")
    elif case == "band":
        Ap, Ai = I.band_pattern(6000, 40)
        coords, kw = None, dict(nb=64, ordering="natural")
    else:
        Ap, Ai, _ = I.random_spd(5000, 0.0008, 11)
        coords, kw = None, dict(nb=48, ordering="rcm")
    n = len(Ap) - 1
    ref = _plan_exports(Plan(n, Ap, Ai, host_threads=1, **kw))
    for t in (2, 3, 8):
        got = _plan_exports(Plan(n, Ap, Ai, host_threads=t, **kw))
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (t, k)
