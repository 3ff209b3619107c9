"""The H*v autotuner: every variant of the fast row kernel computes the same y
bit for bit (and the oracle's on sampled rows), the tuner picks the fastest
variant that fits, and its choice travels through the context cache and the
JSON file to sectors of the same shape."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import sector as osec
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


# fast H*v variants: [0, 5) one up string per block (kernel 2), [5, 10) two up
# strings per block (kernel 3), both x five launch shapes; [10, 16) the
# natural-order kernel (kernel 4) for float and double-float vectors, four or
# two (float) / two or one (double-float) up strings per block x three block
# sizes (float four-row blocks of 1024, 512 and 384 threads)
NV = 16
KERNELS = [2] * 5 + [3] * 5 + [4] * 6


def applicable(m, prec):
    """Variants that apply to a sector of model m in format prec (all of these
    cases have the fast tables)."""
    if prec == "fp64":
        return set(range(5))
    moves = m.n_orb >= 2 and (m.Jsf != 0.0 or m.Jph != 0.0)
    nat = not moves or m.orb0 + m.n_orb == m.n_s
    if prec == "fp32":
        return set(range(10, 16)) if nat else set(range(10))
    return set(range(16)) if nat else set(range(10))


def family(v):
    return 0 if v < 5 else (1 if v < 10 else 2)

CASES = [("Kanamori N_s=12 (6,6)", lambda: W.kanamori(12, seed=0), 6, 6),
         ("Kanamori N_s=13 (6,7)", lambda: W.kanamori(13, seed=3), 6, 7),
         ("AIM N_s=13 (7,6)", lambda: W.aim(13, seed=3), 7, 6),
         ("Kanamori impurity on low sites N_s=13 (6,7)", lambda: W.kanamori(13, seed=3, imp_first=True), 6, 7)]


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("name,mk,nu,nd", CASES, ids=[c[0] for c in CASES])
def test_variants_agree_bitwise_and_tuner_picks_fastest(env, name, mk, nu, nd, prec):
    ed, ctx, torch = env
    m = mk()
    D_dn = len(osec.spin_basis(m.n_s, nd))
    dim = len(osec.spin_basis(m.n_s, nu)) * D_dn
    x = W.random_vector(dim, seed=4)
    sec = ed.ed_sector_create(ctx, m, nu, nd, prec)
    try:
        xd = to_dev(x, prec, ed, torch)
        outs = {}
        nv = NV
        app = applicable(m, prec)
        for v in range(nv):
            try:
                ed.ed_sector_set_variant(sec, v)
            except ed.EdError:
                assert v not in app, v
                continue
            assert v in app, v
            assert ed.ed_sector_get_variant(sec) == v
            y = empty_vec(dim, prec, ed, torch)
            ed.ed_apply_h(sec, xd, y)
            torch.cuda.synchronize()
            outs[v] = y
        # bit for bit within a kernel family; double-float families sum in
        # different orders, within the format's rounding
        base = outs[min(app)]
        for v, y in outs.items():
            first = outs[min(u for u in outs if family(u) == family(v))]
            assert torch.equal(y, first), (v, name, prec)
            if family(v) != family(min(app)):
                yb, bb = to_host(y, prec, dim, ed, torch), to_host(base, prec, dim, ed, torch)
                assert rel_err(yb, bb) <= 1e-13, (v, rel_err(yb, bb))
        rows = np.unique(np.random.default_rng(1).integers(0, dim, 800))
        xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
        ref = osec.apply_rows(m, nu, nd, rows, xin)
        got = to_host(base, prec, dim, ed, torch)[rows]
        assert rel_err(got, ref) <= TOL[prec]

        r = ed.ed_sector_autotune(sec, reps=3)
        assert r.n_candidates == nv
        ms = np.array(r.ms[:nv])
        fit = ms > 0
        assert fit[min(app)]
        assert all(v in app for v in np.nonzero(fit)[0])
        assert r.chosen == int(np.argmin(np.where(fit, ms, np.inf)))
        assert ed.ed_sector_get_variant(sec) == r.chosen
        assert ed.ed_sector_get_info(sec).kernel == r.kernel[r.chosen]
        assert [r.kernel[i] for i in range(nv)] == KERNELS
    finally:
        ed.ed_sector_destroy(sec)


def test_cache_roundtrip_and_other_gpu(env, tmp_path):
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    sec = ed.ed_sector_create(ctx, m, 6, 6, "df64")
    try:
        r = ed.ed_sector_autotune(sec, reps=2)
        chosen = r.chosen
        p = tmp_path / "tune.json"
        ed.ed_tune_cache_save(ctx, str(p))
        doc = json.loads(p.read_text())
        assert doc["format"] == "libedgb-autotune-1" and doc["entries"]
        # a second sector of the same shape in the same context starts tuned
        sec2 = ed.ed_sector_create(ctx, m, 6, 6, "df64")
        assert ed.ed_sector_get_variant(sec2) == chosen
        ed.ed_sector_destroy(sec2)
    finally:
        ed.ed_sector_destroy(sec)
    ctx2 = ed.ed_ctx_create(0)
    try:
        s0 = ed.ed_sector_create(ctx2, m, 6, 6, "df64")
        assert ed.ed_sector_get_variant(s0) == -1
        ed.ed_sector_destroy(s0)
        assert ed.ed_tune_cache_load(ctx2, str(p)) == len(doc["entries"])
        s1 = ed.ed_sector_create(ctx2, m, 6, 6, "df64")
        assert ed.ed_sector_get_variant(s1) == chosen
        ed.ed_sector_destroy(s1)
        # entries measured on another GPU model are skipped
        other = dict(doc, device="some other GPU")
        q = tmp_path / "other.json"
        q.write_text(json.dumps(other))
        assert ed.ed_tune_cache_load(ctx2, str(q)) == 0
        # malformed files are rejected
        for bad in ('{"format": "something else", "device": "x", "entries": []}',
                    json.dumps(dict(doc, entries=[{"key": "k", "variant": 99}])),
                    '{"format": "libedgb-autotune-1", "device": "x", "entries": [{"key": "unterminated'):
            q.write_text(bad)
            with pytest.raises(ed.EdError):
                ed.ed_tune_cache_load(ctx2, str(q))
        with pytest.raises(ed.EdError):
            ed.ed_tune_cache_load(ctx2, str(tmp_path / "missing.json"))
    finally:
        ed.ed_ctx_destroy(ctx2)


def test_nothing_to_tune_and_bad_variants(env):
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    g = ed.ed_sector_create(ctx, m, 6, 6, "df64", ed.ED_SECTOR_GENERIC)
    try:
        r = ed.ed_sector_autotune(g, reps=2)
        assert r.n_candidates == 0 and r.chosen == -1
        assert ed.ed_sector_get_variant(g) == -1
        with pytest.raises(ed.EdError):
            ed.ed_sector_set_variant(g, 0)
    finally:
        ed.ed_sector_destroy(g)
    s = ed.ed_sector_create(ctx, m, 6, 6, "fp64")
    try:
        for bad in (5, 10, NV, -2, 100):
            with pytest.raises(ed.EdError):
                ed.ed_sector_set_variant(s, bad)
        ed.ed_sector_set_variant(s, -1)
        assert ed.ed_sector_get_variant(s) == -1
    finally:
        ed.ed_sector_destroy(s)
