"""The request server: results against the oracle, the same result alone and
in a mix (continuous batching), HBM-footprint admission, poll semantics."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import sector as osec, spectrum, greens as og
from tests._gpu import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


_poll_energies = {}   # ticket -> (status, ed_result, G) as polled


def wait_all(ed, srv, tickets, timeout=300.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            done, res, G = ed.ed_poll(srv, t)
            if done:
                out[t] = (res.status, res.E0, res.iters, G, res.latency_ms)
                _poll_energies[t] = (res.status, res, G)
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.002)
    return out


def request_set():
    reqs = []
    for i, ns in enumerate((8, 9, 10, 11, 12, 10, 9)):
        reqs.append((W.kanamori(ns, seed=100 + i), (ns + 1) // 2, ns // 2))
    return reqs


# Tolerances against the oracle per vector format: ground energy (relative) and
# max |G - G_oracle| over the Matsubara points.  FP64 and DF64 carry the
# spec bounds (eigenvalues 1e-10, G 1e-8).  FP32 vectors round every stored
# element to 2^-24 relative, so the ground energy is held to the 1e-6 relative
# target for the FP32-vector form; G is built from float vectors (phi = c+ psi
# and the Lanczos vectors of the continued fraction), whose coefficients carry
# errors of a few 1e-7 relative, and |G| <= 1/w_0 = beta/pi ~ 12.7 here: 2e-5.
SERVE_TOL = {"fp64": (1e-10, 1e-8), "df64": (1e-10, 1e-8), "fp32": (1e-6, 2e-5)}
# Lanczos residual tolerance of the server per format: the three-vector
# recurrence on float vectors loses orthogonality early and its residual
# estimate does not reach 1e-11; 1e-7 still gives eigenvalues to ~1e-13 (the
# eigenvalue error is quadratic in the residual).
LZ_TOL = {"fp64": 1e-11, "df64": 1e-11, "fp32": 1e-7}


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_server_results_match_oracle_and_are_mix_invariant(env, prec):
    ed, ctx, torch = env
    beta, nw, depth = 40.0, 256, 60
    e_tol, g_tol = SERVE_TOL[prec]
    reqs = request_set()
    srv = ed.ed_server_create(ctx, max_active=4, prec=prec, tol=LZ_TOL[prec], max_iter=400, cf_depth=depth, n_w=nw,
                              beta=beta)
    try:
        # request 0 alone
        t_alone = ed.ed_submit(srv, reqs[0][0], reqs[0][1], reqs[0][2])
        alone = wait_all(ed, srv, [t_alone])[t_alone]
        # the same request again, now arriving in the middle of a mix
        ts = [ed.ed_submit(srv, m, nu, nd) for (m, nu, nd) in reqs[1:4]]
        t_mix = ed.ed_submit(srv, reqs[0][0], reqs[0][1], reqs[0][2])
        ts += [ed.ed_submit(srv, m, nu, nd) for (m, nu, nd) in reqs[4:]]
        res = wait_all(ed, srv, ts + [t_mix])
        mix = res[t_mix]
        assert alone[0] == 0 and mix[0] == 0
        assert alone[1] == mix[1]                      # bit for bit
        assert np.array_equal(alone[3], mix[3])
        # every request against the oracle: ground energy and G
        for (m, nu, nd), t in zip(reqs[1:4] + reqs[4:], ts):
            st, E0, iters, G, lat = res[t]
            assert st == 0
            H = osec.build_csr(m, nu, nd)
            w, v = spectrum.lowest(H, 1, vectors=True)
            assert abs(E0 - w[0]) <= e_tol * abs(w[0]), (m.n_s, E0, w[0])
            Gref = og.greens_cf(m, [(nu, nd, w[0], v[:, 0])], beta, nw, m.orb0, 0, depth=depth)
            assert np.max(np.abs(G - Gref)) <= g_tol, (m.n_s, np.max(np.abs(G - Gref)))
        stats = ed.ed_server_get_stats(srv)
        assert stats.max_active_seen >= 2          # requests overlapped on the device
        assert stats.failed == 0
    finally:
        ed.ed_server_destroy(srv)


def test_server_admission_budget_and_errors(env):
    ed, ctx, torch = env
    reqs = request_set()
    budget = 96 * 1024 * 1024 + 200 * 1024 * 1024   # about two of these requests at once
    srv = ed.ed_server_create(ctx, hbm_budget=budget, max_active=16, prec="fp64", tol=1e-10, cf_depth=30, n_w=32)
    try:
        ts = [ed.ed_submit(srv, m, nu, nd) for (m, nu, nd) in reqs]
        seen = 0
        t0 = time.time()
        while True:
            st = ed.ed_server_get_stats(srv)
            assert st.bytes_in_flight <= budget
            seen = max(seen, st.active)
            if st.done + st.failed == len(ts):
                break
            assert time.time() - t0 < 300
            time.sleep(0.001)
        res = wait_all(ed, srv, ts)
        assert all(r[0] == 0 for r in res.values())
        # latency and queue-time percentiles over the finished requests, as
        # numpy's linear interpolation of the times the results carry
        st = ed.ed_server_get_stats(srv)
        assert st.n_latency == len(ts) and st.queued == 0 and st.active == 0
        lat = [_poll_energies[t][1].latency_ms for t in ts]
        wait = [_poll_energies[t][1].queue_ms for t in ts]
        for got, ref in ((st.latency_p50_ms, np.percentile(lat, 50)), (st.latency_p99_ms, np.percentile(lat, 99)),
                         (st.queue_p50_ms, np.percentile(wait, 50)), (st.queue_p99_ms, np.percentile(wait, 99))):
            assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)
        assert 0 < st.latency_p50_ms <= st.latency_p99_ms <= max(lat)
        # a request larger than the whole budget is refused at submission
        big = W.kanamori(16, seed=1)
        with pytest.raises(ed.EdError) as e:
            ed.ed_submit(srv, big, 8, 8)
        assert e.value.status == ed.ED_ERR_OOM
        # collected and unknown tickets
        with pytest.raises(ed.EdError):
            ed.ed_poll(srv, ts[0])
        with pytest.raises(ed.EdError):
            ed.ed_poll(srv, 10 ** 9)
    finally:
        ed.ed_server_destroy(srv)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_server_k_lowest_states_match_oracle_and_are_mix_invariant(env, prec):
    """k = 4 lowest states per request (thick restart on a server worker thread)
    and G from all four with Boltzmann weights at beta = 40 (Sec. 4 keeps the
    states above a 1e-5 weight): energies and G against the oracle, and the
    same request alone and in a mix of k = 1 and k = 4 requests, bit for bit."""
    ed, ctx, torch = env
    beta, nw, depth, k = 40.0, 128, 50, 4
    e_tol, g_tol = SERVE_TOL[prec]
    reqs = request_set()[:5]
    srv = ed.ed_server_create(ctx, max_active=4, prec=prec, tol=LZ_TOL[prec], max_iter=3000, cf_depth=depth,
                              n_w=nw, beta=beta)
    try:
        m0, nu0, nd0 = reqs[2]
        t_alone = ed.ed_submit(srv, m0, nu0, nd0, k=k)
        alone = wait_all(ed, srv, [t_alone])
        ts = [ed.ed_submit(srv, m, nu, nd, k=(k if i % 2 == 0 else 1)) for i, (m, nu, nd) in enumerate(reqs)]
        res = wait_all(ed, srv, ts)
        mix = res[ts[2]]
        assert alone[t_alone][0] == 0 and mix[0] == 0
        assert alone[t_alone][1] == mix[1]
        assert np.array_equal(alone[t_alone][3], mix[3])
        for i, ((m, nu, nd), t) in enumerate(zip(reqs, ts)):
            st, E0, iters, G, lat = res[t]
            assert st == 0, (i, st)
            _, r, _ = _poll_energies[t]
            kk = k if i % 2 == 0 else 1
            H = osec.build_csr(m, nu, nd)
            w, v = spectrum.lowest(H, kk, vectors=True)
            assert r.n_E == kk
            E = np.array(r.E[:kk])
            assert np.max(np.abs(E - w) / np.abs(w)) <= e_tol, (m.n_s, E, w)
            Gref = og.greens_cf(m, [(nu, nd, w[j], v[:, j]) for j in range(kk)], beta, nw, m.orb0, 0, depth=depth)
            assert np.max(np.abs(G - Gref)) <= g_tol, (m.n_s, np.max(np.abs(G - Gref)))
        assert ed.ed_server_get_stats(srv).failed == 0
    finally:
        ed.ed_server_destroy(srv)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_server_packs_small_requests(env, prec):
    """Requests whose sector has at most pack_dim states are solved in packs
    (one batched Lanczos over all their sectors per step, Ritz vectors from the
    stored basis, then each G).  Energies and G against the oracle; a request
    alone (a pack of one) and in a pack of six with other models, k = 1 and
    k = 4 requests in separate packs, and an unpacked larger request at the
    same time, bit for bit."""
    ed, ctx, torch = env
    beta, nw, depth = 40.0, 128, 50
    e_tol, g_tol = SERVE_TOL[prec]
    small = [(W.kanamori(ns, seed=200 + i), (ns + 1) // 2, ns // 2) for i, ns in enumerate((8, 9, 10, 11, 9, 10))]
    big = (W.kanamori(12, seed=300), 6, 6)                        # 853,776 states: not packed
    srv = ed.ed_server_create(ctx, max_active=4, prec=prec, tol=LZ_TOL[prec], max_iter=3000, cf_depth=depth,
                              n_w=nw, beta=beta, pack_dim=250_000)
    try:
        t_alone = ed.ed_submit(srv, *small[3], k=4)
        alone = wait_all(ed, srv, [t_alone])[t_alone]
        t_big = ed.ed_submit(srv, *big, k=1)
        ts = [ed.ed_submit(srv, m, nu, nd, k=(4 if i < 4 else 1)) for i, (m, nu, nd) in enumerate(small)]
        res = wait_all(ed, srv, ts + [t_big])
        mix = res[ts[3]]
        assert alone[0] == 0 and mix[0] == 0
        assert alone[1] == mix[1] and np.array_equal(alone[3], mix[3])
        assert _poll_energies[t_alone][1].E[:4] == _poll_energies[ts[3]][1].E[:4]
        for i, ((m, nu, nd), t) in enumerate(zip(small + [big], ts + [t_big])):
            st, E0, iters, G, lat = res[t]
            assert st == 0, (i, st)
            kk = 4 if i < 4 else 1
            H = osec.build_csr(m, nu, nd)
            w, v = spectrum.lowest(H, kk, vectors=True)
            E = np.array(_poll_energies[t][1].E[:kk])
            assert np.max(np.abs(E - w) / np.abs(w)) <= e_tol, (m.n_s, E, w)
            Gref = og.greens_cf(m, [(nu, nd, w[j], v[:, j]) for j in range(kk)], beta, nw, m.orb0, 0, depth=depth)
            assert np.max(np.abs(G - Gref)) <= g_tol, (m.n_s, np.max(np.abs(G - Gref)))
        assert ed.ed_server_get_stats(srv).failed == 0
    finally:
        ed.ed_server_destroy(srv)
