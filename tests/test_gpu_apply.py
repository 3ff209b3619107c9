"""Matrix-free H*v through the C ABI vs the oracle's explicit sector H.

FP64 and DF64: ||y - y_ref|| / ||y_ref|| <= 1e-12 (the FP64 target).
FP32 vectors: compared with the oracle applied to the float-rounded input.
The natural-order float kernel sums each element in float in two passes
(diagonal + down hops, then up hops + spin-flip / pair-hop) with the
coefficients rounded to float, so an element's error is at most about
(n + 3) 2^-24 sum_j |H_ij x_j| for n terms (~1e-6 relative for 15 terms in the
worst case, ~1e-7 typical; the exact first-order bound is checked element by
element below); the double-float-accumulating kernels (the fallback) round
once.  The norm-wise tests allow 1e-6.
Small sectors are checked element by element on every row; large ones (row
lengths that select the row-staged kernel, and the full N_s=15 half-filled
sector the benchmark times) on sampled rows, first/last/ragged rows included.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fock, sector as osec
from tests._gpu import ensure_built, torch_cuda, to_dev, to_host, empty_vec, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "fp32": 1e-6}


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


_CSR = {}


def oracle_csr(name, m, nu, nd):
    if name not in _CSR:
        _CSR[name] = osec.build_csr(m, nu, nd)
    return _CSR[name]


def run_apply(ed, ctx, torch, m, nu, nd, prec, x, flags=0, expect_kernel=None):
    sec = ed.ed_sector_create(ctx, m, nu, nd, prec, flags)
    try:
        if expect_kernel is not None:
            assert ed.ed_sector_get_info(sec).kernel == expect_kernel
        n = len(x)
        xd = to_dev(x, prec, ed, torch)
        yd = empty_vec(n, prec, ed, torch)
        ed.ed_apply_h(sec, xd, yd)
        torch.cuda.synchronize()
        return to_host(yd, prec, n, ed, torch)
    finally:
        ed.ed_sector_destroy(sec)


def input_for(prec, x):
    return x.astype(np.float32).astype(np.float64) if prec == "fp32" else x


FULL = [
    ("C0 AIM N_s=6 (3,3)", lambda: W.aim(6, seed=0), 3, 3),
    ("Kanamori N_s=8 (4,3)", lambda: W.kanamori(8, seed=1), 4, 3),
    ("Kanamori M=2 N_s=7 (3,4)", lambda: W.kanamori(7, seed=5, n_orb=2), 3, 4),
    ("Hubbard ring N_s=10 (5,4) two diagonal chunks", lambda: W.hubbard_cluster(10, tp=0.3), 5, 4),
    ("Hubbard ring N_s=12 (6,6) K=12", lambda: W.hubbard_cluster(12, tp=0.2), 6, 6),
    ("atom (2,1)", lambda: W.atom(3), 2, 1),
    ("dim 1 (0,0)", lambda: W.kanamori(8, seed=2), 0, 0),
    ("dim 1 full (8,8)", lambda: W.kanamori(8, seed=2), 8, 8),
    ("D_up 1 (0,3)", lambda: W.kanamori(8, seed=2), 0, 3),
    ("D_dn 1 (5,8)", lambda: W.kanamori(8, seed=2), 5, 8),
    ("Kanamori 4 orbitals N_s=9 (4,5)", lambda: W.kanamori(9, seed=4, n_orb=4), 4, 5),
    ("Kanamori impurity on low sites N_s=8 (4,3)", lambda: W.kanamori(8, seed=1, imp_first=True), 4, 3),
    ("AIM impurity on low site N_s=6 (3,3)", lambda: W.aim(6, seed=0, imp_first=True), 3, 3),
    # fast row kernels (D_dn >= 512): 1716 down strings = 53 full groups of 32
    # plus 20; 78 and 13 up strings leave ragged tiles of 2- and 4-row blocks
    ("Kanamori N_s=13 (2,6) ragged row tiles", lambda: W.kanamori(13, seed=3), 2, 6),
    ("Kanamori N_s=13 (1,6) one-row tail", lambda: W.kanamori(13, seed=3), 1, 6),
    ("AIM N_s=13 (3,6)", lambda: W.aim(13, seed=4), 3, 6),
    ("C1 Kanamori N_s=12 (6,6) full", lambda: W.kanamori(12, seed=0), 6, 6),
]


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("name,mk,nu,nd", FULL, ids=[c[0] for c in FULL])
def test_apply_full_sector(env, name, mk, nu, nd, prec):
    ed, ctx, torch = env
    m = mk()
    H = oracle_csr(name, m, nu, nd)
    x = W.random_vector(H.shape[0], seed=1)
    xin = input_for(prec, x)
    y = run_apply(ed, ctx, torch, m, nu, nd, prec, x)
    ref = H @ xin
    assert rel_err(y, ref) <= TOL[prec], rel_err(y, ref)
    if prec == "fp64":
        assert np.max(np.abs(y - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def sample_rows(dim, D_dn, k=2500, seed=3):
    rng = np.random.default_rng(seed)
    rows = set(rng.integers(0, dim, k).tolist())
    rows |= {0, 1, D_dn - 1, D_dn, dim - 1, dim - 2, dim // 2, (dim // D_dn - 1) * D_dn}
    return np.array(sorted(r for r in rows if 0 <= r < dim))


# (name, model, n_up, n_dn, kernel chosen by default: 0 flat, 1 row-staged generic, 2 fast rows;
# the fast path runs two rows per block (kernel 3) for FP32 vectors)
SAMPLED = [
    ("C1 Kanamori N_s=12 (6,6)", lambda: W.kanamori(12, seed=0), 6, 6, 2),
    ("Kanamori N_s=13 (6,7)", lambda: W.kanamori(13, seed=3), 6, 7, 2),
    ("AIM N_s=13 (7,6)", lambda: W.aim(13, seed=3), 7, 6, 2),
    ("Kanamori 2 orbitals N_s=13 (7,7)", lambda: W.kanamori(13, seed=8, n_orb=2), 7, 7, 2),
    ("Hubbard ring N_s=13 (7,6) K=13", lambda: W.hubbard_cluster(13, tp=0.1), 7, 6, 1),
    ("Kanamori impurity on low sites N_s=13 (6,7)", lambda: W.kanamori(13, seed=3, imp_first=True), 6, 7, 2),
    ("Kanamori 4 orbitals N_s=14 (7,5)", lambda: W.kanamori(14, seed=5, n_orb=4), 7, 5, 2),
    ("Kanamori N_s=13 (1,6) odd row count", lambda: W.kanamori(13, seed=3), 1, 6, 2),
    ("AIM N_s=13 (3,6) two-row pairs", lambda: W.aim(13, seed=4), 3, 6, 2),
]


def fast_kernel(kern, prec, m=None):
    """Kernel id ed_sector_get_info reports by default: float sectors on the
    fast path run the natural-order kernel (4), or the two-row kernel (3) where
    spin-flip / pair-hop moves exist with the impurity orbitals off the top
    sites; FP64 and double-float sectors the one-row window kernel (2)."""
    if kern != 2 or prec != "fp32":
        return kern
    moves = m is not None and m.n_orb >= 2 and (m.Jsf != 0.0 or m.Jph != 0.0)
    return 3 if moves and m.orb0 + m.n_orb != m.n_s else 4


@pytest.mark.parametrize("generic", [False, True], ids=["default", "generic"])
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("name,mk,nu,nd,kern", SAMPLED, ids=[c[0] for c in SAMPLED])
def test_apply_sampled_rows(env, name, mk, nu, nd, kern, prec, generic):
    ed, ctx, torch = env
    m = mk()
    D_dn = len(osec.spin_basis(m.n_s, nd))
    dim = len(osec.spin_basis(m.n_s, nu)) * D_dn
    x = W.random_vector(dim, seed=2)
    xin = input_for(prec, x)
    flags = ed.ED_SECTOR_GENERIC if generic else 0
    want = (1 if D_dn >= 1024 else 0) if generic else fast_kernel(kern, prec, m)
    if prec == "fp32" and want == 1 and D_dn * 4 > 96 * 1024:
        want = 0
    y = run_apply(ed, ctx, torch, m, nu, nd, prec, x, flags, expect_kernel=want)
    rows = sample_rows(dim, D_dn)
    ref = osec.apply_rows(m, nu, nd, rows, xin)
    assert rel_err(y[rows], ref) <= TOL[prec], rel_err(y[rows], ref)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_apply_n15_half_filling_sampled(env, prec):
    """The N_s=15 (7,8) sector (dim 41,409,225) in the launch configuration the
    benchmark times (fast row kernel), checked on sampled rows."""
    ed, ctx, torch = env
    m = W.kanamori(15, seed=0)
    nu, nd = 7, 8
    dim = 6435 * 6435
    x = W.random_vector(dim, seed=1)
    xin = input_for(prec, x)
    y = run_apply(ed, ctx, torch, m, nu, nd, prec, x, expect_kernel=fast_kernel(2, prec, m))
    rows = sample_rows(dim, 6435, k=1500)
    ref = osec.apply_rows(m, nu, nd, rows, xin)
    assert rel_err(y[rows], ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_apply_n15_window_edges(env, prec):
    """N_s=15 (7,8): every element of the row kernel's 128-string windows that
    span two impurity patterns (spin-flip / pair-hop shifts differ inside the
    window) and of the padded last window (6435 = 50*128 + 35), on the first,
    the last and 40 random up rows, checked against the oracle."""
    ed, ctx, torch = env
    m = W.kanamori(15, seed=0)
    nu, nd = 7, 8
    dbas = osec.spin_basis(15, nd)
    D = len(dbas)
    dim = D * D
    pat = (dbas >> np.uint64(15 - 3)).astype(np.int64)  # impurity orbitals are the top sites
    starts = np.nonzero(np.diff(pat))[0] + 1            # first rank of each new pattern block
    wins = sorted({int(b) // 128 for b in starts if int(b) % 128} | {(D - 1) // 128})
    ds = np.concatenate([np.arange(w * 128, min(D, (w + 1) * 128)) for w in wins])
    assert len(wins) >= 2 and D % 128 != 0
    us = np.unique(np.concatenate([[0, D - 1], np.random.default_rng(11).integers(0, D, 40)]))
    rows = (us[:, None] * D + ds[None, :]).ravel()
    x = W.random_vector(dim, seed=7)
    xin = input_for(prec, x)
    y = run_apply(ed, ctx, torch, m, nu, nd, prec, x, expect_kernel=fast_kernel(2, prec, m))
    ref = osec.apply_rows(m, nu, nd, rows, xin)
    assert rel_err(y[rows], ref) <= TOL[prec], rel_err(y[rows], ref)


def test_apply_csr_variant(env):
    ed, ctx, torch = env
    for m, nu, nd in ((W.aim(6), 3, 3), (W.kanamori(10, seed=6), 5, 5)):
        H = osec.build_csr(m, nu, nd)
        sec = ed.ed_sector_create(ctx, m, nu, nd, "fp64", ed.ED_SECTOR_CSR)
        try:
            x = W.random_vector(H.shape[0], seed=4)
            xd = torch.from_numpy(x).cuda()
            y1 = torch.empty_like(xd)
            y2 = torch.empty_like(xd)
            ed.ed_apply_h_csr(sec, xd, y1)
            ed.ed_apply_h(sec, xd, y2)
            torch.cuda.synchronize()
            ref = H @ x
            assert rel_err(y1.cpu().numpy(), ref) <= 1e-12
            assert rel_err(y2.cpu().numpy(), y1.cpu().numpy()) <= 1e-13
        finally:
            ed.ed_sector_destroy(sec)


def test_apply_is_deterministic_and_symmetric(env):
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    sec = ed.ed_sector_create(ctx, m, 6, 6, "fp64")
    try:
        n = 924 * 924
        a = torch.from_numpy(W.random_vector(n, 5)).cuda()
        b = torch.from_numpy(W.random_vector(n, 6)).cuda()
        ha, hb, ha2 = torch.empty_like(a), torch.empty_like(a), torch.empty_like(a)
        ed.ed_apply_h(sec, a, ha)
        ed.ed_apply_h(sec, b, hb)
        ed.ed_apply_h(sec, a, ha2)
        torch.cuda.synchronize()
        assert torch.equal(ha, ha2)
        # <b, H a> = <H b, a>
        lhs = float(torch.dot(b, ha))
        rhs = float(torch.dot(hb, a))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
        with pytest.raises(ed.EdError):
            ed.ed_apply_h(sec, a, a)
    finally:
        ed.ed_sector_destroy(sec)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_apply_host_buffers_pipeline(env, prec):
    """ed_apply_h_host: n_vec vectors from pinned host memory, copies pipelined
    with the applies on internal streams, gives y bit for bit equal to
    ed_apply_h on device copies of the same vectors, for n_vec = 3 (both
    device buffers reused), 1 and 0, from pinned and from pageable memory."""
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    sec = ed.ed_sector_create(ctx, m, 6, 5, prec)
    try:
        dim = ed.ed_sector_get_info(sec).dim
        n_vec = 3
        xs = [to_dev(W.random_vector(dim, seed=10 + i), prec, ed, torch) for i in range(n_vec)]
        ref = []
        for xd in xs:
            yd = torch.empty_like(xd)
            ed.ed_apply_h(sec, xd, yd)
            ref.append(yd.cpu())
        torch.cuda.synchronize()
        hx = torch.cat([xd.cpu() for xd in xs]).pin_memory()
        hy = torch.full_like(hx, float("nan")).pin_memory()
        ed.ed_apply_h_host(sec, n_vec, hx, hy)
        per = hx.numel() // n_vec
        for i in range(n_vec):
            assert torch.equal(hy[i * per:(i + 1) * per], ref[i]), i
        hy1 = torch.full_like(hx[:per], float("nan")).pin_memory()
        ed.ed_apply_h_host(sec, 1, hx[per:2 * per], hy1)
        assert torch.equal(hy1, ref[1])
        ed.ed_apply_h_host(sec, 0, hx, hy1)            # nothing to do
        assert torch.equal(hy1, ref[1])
        npx = hx[2 * per:].numpy().copy()               # pageable numpy buffers
        npy = np.full_like(npx, np.nan)
        ed.ed_apply_h_host(sec, 1, npx, npy)
        assert np.array_equal(npy, ref[2].numpy())
        with pytest.raises(ed.EdError):
            ed.ed_apply_h_host(sec, 1, None, hy1)
    finally:
        ed.ed_sector_destroy(sec)


def density_term_magnitude(m, nu, nd):
    """Per basis state, the sum of |coefficient| over the density terms of H that
    are on in it (T_ii n_is, U_i n_iu n_id, (U' - J delta_ss') n_ms n_m's'): a
    bound on |e_up| + |e_dn| + |W|, the three pieces the float kernel rounds to
    float and adds to form the diagonal (e_up of the up string, e_dn of the down
    string, W of their orbital occupations)."""
    def density(ops):
        return all(ops[k][0] == ops[k + 1][0] and ops[k][1] and not ops[k + 1][1] for k in range(0, len(ops), 2))
    terms = [(abs(c), ops) for c, ops in fock.hamiltonian_terms(m) if density(ops)]
    return osec.build_csr(m, nu, nd, terms=terms).diagonal()


ELEMENTWISE = [("Kanamori N_s=12 (6,6)", lambda: W.kanamori(12, seed=0), 6, 6),
               ("Kanamori N_s=13 (6,7)", lambda: W.kanamori(13, seed=3), 6, 7),
               ("AIM N_s=12 (6,6)", lambda: W.aim(12, seed=2), 6, 6)]


@pytest.mark.parametrize("name,mk,nu,nd", ELEMENTWISE, ids=[c[0] for c in ELEMENTWISE])
def test_fp32_float_sums_within_elementwise_bound(env, name, mk, nu, nd):
    """The natural-order float kernel's error, element by element, against the
    first-order bound of its arithmetic: pass A (diagonal, then n_A - 1 down
    hops) and pass B (n_B up hops and spin-flip / pair-hop terms) are FMA chains
    in float with the coefficients rounded to float (one rounding each), the
    diagonal is formed from three float pieces by two additions and multiplies
    x_i once, and y = fl(A + B):
      |y_i - (Hx)_i| <= u [(n_A + 1) sum_A |H_ij x_j| + 4 S_i |x_i|
                           + (n_B + 1) sum_B |H_ij x_j| + |(Hx)_i|],
    u = 2^-24, sum_A over the row's own up string, sum_B over the others, S_i
    the density-term magnitude of state i, with a 1% allowance for second-order
    terms."""
    ed, ctx, torch = env
    m = mk()
    H = oracle_csr(name, m, nu, nd)
    n = H.shape[0]
    D_dn = len(osec.spin_basis(m.n_s, nd))
    x = input_for("fp32", W.random_vector(n, seed=7))
    ref = H @ x
    y = run_apply(ed, ctx, torch, m, nu, nd, "fp32", x, expect_kernel=4)
    coo = H.tocoo()
    own = (coo.row // D_dn) == (coo.col // D_dn)
    A = sp.csr_matrix((np.abs(coo.data[own]), (coo.row[own], coo.col[own])), shape=H.shape)
    B = sp.csr_matrix((np.abs(coo.data[~own]), (coo.row[~own], coo.col[~own])), shape=H.shape)
    n_A = np.diff(A.indptr) + 1          # entries of the row (diagonal included), plus one for duplicates
    n_B = np.diff(B.indptr) + 1
    S = density_term_magnitude(m, nu, nd)
    ax = np.abs(x)
    u = 2.0 ** -24
    bound = u * ((n_A + 1) * (A @ ax) + 4 * S * ax + (n_B + 1) * (B @ ax) + np.abs(ref)) * 1.01
    err = np.abs(y - ref)
    assert np.all(err <= bound), (name, int(np.argmax(err / np.maximum(bound, 1e-300))), float(np.max(err / bound)))
    # the bound is not vacuous: the worst element uses a good part of it
    assert np.max(err / bound) > 0.02


def test_fp32_vectors_with_double_float_sums(env):
    """ED_SECTOR_ACC_DF: float vectors whose H*v keeps double-float sums (the
    two-row kernel) round each element once, so every element is within 2^-24
    relative of the oracle applied to the float input; the default
    (natural-order kernel, float sums) stays within its stated bound."""
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    H = oracle_csr("C1 Kanamori N_s=12 (6,6) full", m, 6, 6)
    x = W.random_vector(H.shape[0], seed=1)
    ref = H @ input_for("fp32", x)
    y_df = run_apply(ed, ctx, torch, m, 6, 6, "fp32", x, ed.ED_SECTOR_ACC_DF, expect_kernel=3)
    # one rounding to float, plus the double-float sum's own error (~2^-46 of sum |H_ij x_j|)
    scale = abs(H) @ np.abs(input_for("fp32", x))
    assert np.all(np.abs(y_df - ref) <= 2.0 ** -24 * np.abs(ref) + 2.0 ** -40 * scale)
    y_nat = run_apply(ed, ctx, torch, m, 6, 6, "fp32", x, expect_kernel=4)
    assert rel_err(y_nat, ref) <= 1e-6
