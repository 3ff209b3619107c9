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


NV = 10  # fast H*v variants: one or two up strings per block x five launch shapes

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
        for v in range(nv):
            try:
                ed.ed_sector_set_variant(sec, v)
            except ed.EdError:
                assert prec == "fp64" and v >= nv // 2   # two-row variants exist for DF64 and FP32 only
                continue
            assert ed.ed_sector_get_variant(sec) == v
            y = empty_vec(dim, prec, ed, torch)
            ed.ed_apply_h(sec, xd, y)
            torch.cuda.synchronize()
            outs[v] = y
        base = outs[0]
        for v, y in outs.items():
            assert torch.equal(y, base), (v, name, prec)
        rows = np.unique(np.random.default_rng(1).integers(0, dim, 800))
        xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
        ref = osec.apply_rows(m, nu, nd, rows, xin)
        got = to_host(base, prec, dim, ed, torch)[rows]
        assert rel_err(got, ref) <= TOL[prec]

        r = ed.ed_sector_autotune(sec, reps=3)
        assert r.n_candidates == nv
        ms = np.array(r.ms[:nv])
        fit = ms > 0
        assert fit[:nv // 2].any()
        if prec == "fp64":
            assert not fit[nv // 2:].any()
        assert r.chosen == int(np.argmin(np.where(fit, ms, np.inf)))
        assert ed.ed_sector_get_variant(sec) == r.chosen
        assert ed.ed_sector_get_info(sec).kernel == r.kernel[r.chosen]
        assert [r.kernel[i] for i in range(nv)] == [2] * (nv // 2) + [3] * (nv // 2)
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
        for bad in (NV // 2, NV, -2, 100):
            with pytest.raises(ed.EdError):
                ed.ed_sector_set_variant(s, bad)
        ed.ed_sector_set_variant(s, -1)
        assert ed.ed_sector_get_variant(s) == -1
    finally:
        ed.ed_sector_destroy(s)
