// Request server for impurity solves (the per-iteration workload of the DMFT
// loop, Sec. 2: each iteration diagonalises a new impurity Hamiltonian for its
// lowest state and forms G(i w_n), Eq. 3).
//
// Continuous batching: a server thread admits queued requests whenever the
// HBM budget and the slot limit allow, and advances every admitted request by
// a few Lanczos steps per pass, each request on its own CUDA stream with its
// own scratch, so the work of requests that arrived at different times
// overlaps on the device.  A request is a resumable state machine:
//
//   GS    ground state of its sector, three-vector Lanczos (fused kernels,
//         one CUDA graph per step and buffer rotation), convergence checked
//         asynchronously (tridiagonal solve on the device, event polled)
//   VEC   Ritz vector by regenerating the same Krylov vectors
//   CF+   c+ psi into the N+1 sector, `depth` Lanczos steps (coefficients)
//   CF-   c psi into the N-1 sector, same
//   EVAL  continued fractions on n_w Matsubara points, copied to the host
//
// Each request's kernels touch only its own buffers, so a result is the same
// bit for bit whether the request ran alone or in a mix.
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>

#include "lanczos_kernels.h"

namespace ed {

int trlan_run(Sector* s, const ed_trlan_opts* o, double* evals, void* evecs, ed_trlan_info* info,
              cudaStream_t st);
int greens_cf_run(Ctx* ctx, const ed_model* m, int prec, int n_states, const ed_state* states, double beta,
                  int n_w, const double* z, int orbital, int spin, int depth, double boltz_cut, double* G,
                  double* coeffs, cudaStream_t st);
int batch_solve_pack(Ctx* ctx, int prec, int n, const ed_model* const* models, const int* n_up, const int* n_dn,
                     const ed_lanczos_opts* o, uint32_t chunk, double* evals, int* iters, int* conv,
                     void* const* ritz);
int greens_accumulate(double2* dG, int n_w, double beta, const double* da, const double* db, int L, double n2,
                      const double* dE, int n_states, int nu, int sgn, cudaStream_t st);

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Resumable three-vector Lanczos on one sector, on one stream, with its own
// scratch; steps are replays of one of three captured graphs (the buffer
// rotation j % 3), the step index lives on the device.
template <class V>
struct Run3 {
  Sector* s = nullptr;
  Ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  uint64_t n = 0;
  int mmax = 0;
  V* Q[3] = {nullptr, nullptr, nullptr};
  V* Y = nullptr;
  V* v0 = nullptr;
  double* partial = nullptr;
  Coefs c{};
  char* cbuf = nullptr;
  size_t cbytes = 0;
  uint32_t sgrid = 0;
  int np_apply = 0;
  cudaGraphExec_t g[3] = {nullptr, nullptr, nullptr};
  int launched = 0;
  std::vector<std::pair<void*, size_t>> allocs;

  template <class T>
  int alloc(T** p, size_t count) {
    int r = dev_alloc(ctx, reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (r == ED_OK) allocs.push_back({(void*)*p, std::max<size_t>(count, 1) * sizeof(T)});
    return r;
  }
  void release() {
    for (int i = 0; i < 3; ++i)
      if (g[i]) cudaGraphExecDestroy(g[i]);
    for (auto& a : allocs) dev_free(ctx, a.first, a.second);
    allocs.clear();
  }
  ~Run3() { release(); }

  V* q(int j) { return Q[((j % 3) + 3) % 3]; }

  int apply_dot_launch(const V* x, V* y) {
    if (s->fast.ok) return apply_fast(s, x, y, st, partial, &np_apply);
    ED_TRY(apply_h(s, x, y, st));
    k_dot<V><<<sgrid, kRedThreads, 0, st>>>(x, y, n, partial);
    ED_LAUNCH_CHECK();
    np_apply = (int)sgrid;
    return ED_OK;
  }

  // Allocate, copy the start vector (or draw one), normalise, capture the step graphs.
  int init(Sector* sec, Ctx* cx, cudaStream_t stream, int max_steps, const V* start, uint64_t seed, int k,
           double thr) {
    s = sec;
    ctx = cx;
    st = stream;
    n = s->dim;
    mmax = max_steps;
    for (int i = 0; i < 3; ++i) ED_TRY(alloc(&Q[i], n));
    ED_TRY(alloc(&Y, n));
    ED_TRY(alloc(&v0, n));
    sgrid = (uint32_t)std::min<uint64_t>((n + kRedThreads - 1) / kRedThreads, (uint64_t)ctx->num_sms * 8);
    if (sgrid == 0) sgrid = 1;
    ED_TRY(alloc(&partial, std::max<uint64_t>(sgrid, (uint64_t)ctx->num_sms * 8)));
    cbytes = coef_bytes(mmax, std::max(k, 1)) + 8 * 1024 + (size_t)(mmax + 2) * 64 * std::max(k, 1);
    ED_TRY(alloc(&cbuf, cbytes));
    Carve cv{cbuf};
    c = carve_coefs(cv, mmax);
    k_init_coefs<<<1, 256, 0, st>>>(c, mmax + 2);
    if (start) {
      ED_TRY_CUDA(cudaMemcpyAsync(Q[0], start, n * sizeof(V), cudaMemcpyDeviceToDevice, st));
    } else {
      uint32_t vg = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 16);
      k_random<V><<<vg ? vg : 1, 256, 0, st>>>(Q[0], n, seed);
    }
    ED_TRY_CUDA(cudaMemcpyAsync(v0, Q[0], n * sizeof(V), cudaMemcpyDeviceToDevice, st));
    k_dot<V><<<sgrid, kRedThreads, 0, st>>>(Q[0], Q[0], n, partial);
    k_finish<<<1, kRedThreads, 0, st>>>(partial, (int)sgrid, OP_SIGMA0, 0, c, 0.0);
    ED_LAUNCH_CHECK();
    for (int ph = 0; ph < 3; ++ph) {
      cudaGraph_t graph = nullptr;
      ED_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int r = apply_dot_launch(Q[ph], Y);
      k_finish<<<1, kRedThreads, 0, st>>>(partial, np_apply, OP_ALPHA_Q, -1, c, 0.0);
      k_lz_step<V><<<sgrid, kRedThreads, 0, st>>>(Y, Q[ph], Q[(ph + 2) % 3], Q[(ph + 1) % 3], n, c, -1, partial);
      k_finish<<<1, kRedThreads, 0, st>>>(partial, (int)sgrid, OP_BETA_Q, -2, c, thr);
      k_step_inc<<<1, 1, 0, st>>>(c.step);
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (r != ED_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
      }
      if (ce != cudaSuccess) {
        set_error("step graph capture failed: %s", cudaGetErrorString(ce));
        return ED_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&g[ph], graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        set_error("step graph instantiation failed: %s", cudaGetErrorString(ce));
        return ED_ERR_CUDA;
      }
    }
    launched = 0;
    return ED_OK;
  }

  int launch_step() {
    ED_TRY_CUDA(cudaGraphLaunch(g[launched % 3], st));
    ++launched;
    return ED_OK;
  }
};

enum Phase { PH_QUEUED = 0, PH_GS, PH_GS_CHECK, PH_VEC, PH_CF, PH_CF_WAIT, PH_EVAL_WAIT, PH_WORK, PH_PACK, PH_DONE,
             PH_FAILED };

// Packs of small requests: at most kMaxPack requests, Lanczos steps capped at
// kPackIter (the basis holds them all), work items of kPackChunk elements.
constexpr int kMaxPack = 64;
constexpr int kPackIter = 400;
constexpr uint32_t kPackChunk = 4096;

// Thick-restart basis of a k > 1 request: max(4k + 8, 20) vectors, at most 64.
inline int tr_basis(int k) { return std::min(std::max(4 * k + 8, 20), 64); }

template <class V>
struct Req {
  uint64_t ticket = 0;
  std::vector<double> T, U;
  ed_model model{};
  int n_up = 0, n_dn = 0, want_G = 1, orbital = 0, spin = 0, k = 1;
  bool packed = false;      // solved in a pack of small requests
  uint64_t dim = 0;
  Phase phase = PH_QUEUED;
  size_t footprint = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = ED_OK;
  std::string err;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::unique_ptr<Sector> sec, sec_cf;
  std::unique_ptr<Run3<V>> gs, cf;
  // GS check
  int m_check = 0, m_final = 0;
  double* h_pin = nullptr;  // pinned host staging
  double E0 = NAN;
  int gs_iters = 0;
  // vector
  V* psi = nullptr;
  double* Sd = nullptr;
  float2* Sf = nullptr;
  double* Sq = nullptr;
  float2* Sqf = nullptr;
  double* theta = nullptr;
  double* resid = nullptr;
  double* twork = nullptr;
  int vec_step = 0;
  // CF
  int cf_part = 0;  // 0 particle, 1 hole
  int cf_steps = 0;
  double2* dG = nullptr;
  double* dE = nullptr;
  double* dab = nullptr;
  std::vector<double> G;
  std::vector<double> Ek;   // lowest energies (k > 1, or E0 alone)
  // k > 1: worker thread with its own sub-context (private reduction scratch)
  std::thread worker;
  std::atomic<bool> wdone{false};
  std::unique_ptr<Ctx> sub;
  std::vector<std::pair<void*, size_t>> allocs;
  Ctx* ctx = nullptr;
  template <class T>
  int alloc(T** p, size_t count) {
    int r = dev_alloc(ctx, reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (r == ED_OK) allocs.push_back({(void*)*p, std::max<size_t>(count, 1) * sizeof(T)});
    return r;
  }
  void release() {
    if (worker.joinable()) worker.join();
    gs.reset();
    cf.reset();
    if (sec) free_sector(sec.get());
    if (sec_cf) free_sector(sec_cf.get());
    sec.reset();
    sec_cf.reset();
    for (auto& a : allocs) dev_free(ctx, a.first, a.second);
    allocs.clear();
    if (sub) free_sub_ctx(sub.get());
    sub.reset();
    if (h_pin) cudaFreeHost(h_pin);
    h_pin = nullptr;
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
    if (st) cudaStreamDestroy(st);
    st = nullptr;
  }
};

}  // namespace

struct ServerBase {
  virtual ~ServerBase() {}
  virtual int submit(const ed_request* r, uint64_t* ticket) = 0;
  virtual int poll(uint64_t ticket, ed_result* res, double* G, int* done) = 0;
  virtual int stats(ed_server_stats* s) = 0;
};

namespace {

template <class V>
struct Server : ServerBase {
  Ctx* ctx;
  ed_server_opts o;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::unique_ptr<Req<V>>> queue;
  std::deque<std::unique_ptr<Req<V>>> pack_q;  // queued small requests
  std::thread pack_th;                          // the running pack's worker
  std::atomic<bool> pack_done{false};
  bool pack_running = false;
  std::vector<Req<V>*> pack_reqs;
  std::vector<std::unique_ptr<Req<V>>> active;
  std::map<uint64_t, std::unique_ptr<Req<V>>> finished;
  std::set<uint64_t> live;  // submitted and not yet collected
  std::atomic<bool> stop{false};
  std::thread th;
  uint64_t next_ticket = 1;
  size_t in_flight_bytes = 0;
  int n_done = 0, n_failed = 0, max_active_seen = 0;
  std::vector<double> lat_ms, wait_ms;  // per finished request: submission to completion / admission

  Server(Ctx* c, const ed_server_opts& op) : ctx(c), o(op) { th = std::thread([this] { loop(); }); }
  ~Server() override {
    stop = true;
    cv.notify_all();
    if (th.joinable()) th.join();
    if (pack_th.joinable()) pack_th.join();
    // workers of k > 1 requests run to the end of their solve (release joins them)
    cudaSetDevice(ctx->device);
    for (auto& r : active) r->release();
    for (auto& kv : finished) kv.second->release();
  }

  size_t estimate(int n_s, int nu, int nd, int k) const {
    auto C = [](int n, int k) -> double {
      if (k < 0 || k > n) return 0;
      double r = 1;
      for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
      return r;
    };
    const double dim = C(n_s, nu) * C(n_s, nd);
    const double dcf = std::max({C(n_s, nu + 1) * C(n_s, nd), C(n_s, nu - 1) * C(n_s, nd),
                                 C(n_s, nu) * C(n_s, nd + 1), C(n_s, nu) * C(n_s, nd - 1)});
    const double eb = (double)elem_bytes(o.prec);
    if (o.pack_dim && dim <= (double)o.pack_dim) {
      // packed: the full Krylov basis and the k Ritz vectors, then the Green's function
      const double steps = std::min<double>((double)std::min(o.max_iter, kPackIter), dim);
      return (size_t)(((steps + 3.0 + k) * (dim + 32.0) + 6.0 * dcf) * eb + 64.0 * 1024 * 1024);
    }
    if (k > 1) {
      // thick-restart basis (m + 2 + keep slots, padded) and the k Ritz vectors,
      // then the Green's function: both neighbour sectors' tables, phi and the
      // four vectors of the coefficient recurrence, plus tables
      const double m = tr_basis(k), keep = (m + k) / 2.0;
      return (size_t)(((m + 2.0 + keep + k) * (dim + 32.0) + 6.0 * dcf) * eb + 96.0 * 1024 * 1024);
    }
    // ground-state run (5 vectors) + psi, then CF run (5 vectors) + phi, tables
    return (size_t)((6.0 * dim + 6.0 * dcf) * eb + 64.0 * 1024 * 1024);
  }

  int submit(const ed_request* r, uint64_t* ticket) override {
    ED_TRY(validate_model(r->model));
    const ed_model* m = r->model;
    if (r->n_up < 0 || r->n_up > m->n_s || r->n_dn < 0 || r->n_dn > m->n_s) ED_INVALID("particle numbers out of range");
    std::unique_ptr<Req<V>> q(new Req<V>());
    q->T.assign(m->T, m->T + m->n_s * m->n_s);
    q->U.assign(m->U_site, m->U_site + m->n_s);
    q->model = *m;
    q->model.T = q->T.data();
    q->model.U_site = q->U.data();
    q->n_up = r->n_up;
    q->n_dn = r->n_dn;
    q->want_G = r->want_G;
    q->orbital = r->orbital;
    q->spin = r->spin;
    q->k = r->k < 1 ? 1 : r->k;
    if (q->k > ED_SERVE_MAX_K) ED_INVALID("k = %d outside 1..%d", r->k, ED_SERVE_MAX_K);
    q->ctx = ctx;
    q->footprint = estimate(m->n_s, r->n_up, r->n_dn, q->k);
    {
      auto C = [](int n, int k) -> uint64_t {
        if (k < 0 || k > n) return 0;
        uint64_t r = 1;
        for (int i = 0; i < k; ++i) r = r * (uint64_t)(n - i) / (uint64_t)(i + 1);
        return r;
      };
      q->dim = C(m->n_s, r->n_up) * C(m->n_s, r->n_dn);
      q->packed = o.pack_dim && q->dim <= o.pack_dim;
    }
    if (o.hbm_budget && q->footprint > o.hbm_budget) {
      set_error("request needs ~%zu bytes, more than the whole server budget %zu", q->footprint, o.hbm_budget);
      return ED_ERR_OOM;
    }
    q->t_submit = now_ms();
    std::lock_guard<std::mutex> lk(mu);
    q->ticket = next_ticket++;
    *ticket = q->ticket;
    live.insert(q->ticket);
    queue.push_back(std::move(q));
    cv.notify_all();
    return ED_OK;
  }

  int poll(uint64_t ticket, ed_result* res, double* G, int* done) override {
    std::lock_guard<std::mutex> lk(mu);
    *done = 0;
    auto it = finished.find(ticket);
    if (it == finished.end()) {
      if (live.count(ticket)) return ED_OK;  // queued, being admitted or running
      ED_INVALID("unknown ticket %llu", (unsigned long long)ticket);
    }
    Req<V>* q = it->second.get();
    *done = 1;
    if (res) {
      res->status = q->status;
      res->E0 = q->E0;
      res->iters = q->gs_iters;
      res->latency_ms = q->t_done - q->t_submit;
      res->queue_ms = q->t_admit - q->t_submit;
      res->n_w = q->want_G ? o.n_w : 0;
      const std::vector<double>& E = q->Ek.empty() ? std::vector<double>(1, q->E0) : q->Ek;
      res->n_E = (int)std::min<size_t>(E.size(), ED_SERVE_MAX_K);
      for (int i = 0; i < ED_SERVE_MAX_K; ++i) res->E[i] = i < res->n_E ? E[i] : NAN;
    }
    if (G && q->want_G && !q->G.empty()) std::memcpy(G, q->G.data(), sizeof(double) * q->G.size());
    int st = q->status;
    if (st != ED_OK) set_error("%s", q->err.c_str());
    finished.erase(it);
    live.erase(ticket);
    return ED_OK;
  }

  int stats(ed_server_stats* s) override {
    std::lock_guard<std::mutex> lk(mu);
    s->queued = (int)queue.size();
    s->active = (int)active.size();
    s->done = n_done;
    s->failed = n_failed;
    s->bytes_in_flight = in_flight_bytes;
    s->max_active_seen = max_active_seen;
    s->n_latency = (int)lat_ms.size();
    s->latency_p50_ms = percentile(lat_ms, 50.0);
    s->latency_p99_ms = percentile(lat_ms, 99.0);
    s->queue_p50_ms = percentile(wait_ms, 50.0);
    s->queue_p99_ms = percentile(wait_ms, 99.0);
    return ED_OK;
  }

  // q-th percentile with linear interpolation between order statistics
  // (position q/100 * (n - 1) in the sorted values); 0 without values
  static double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q / 100.0 * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    if (i + 1 >= v.size()) return v.back();
    return v[i] + (pos - (double)i) * (v[i + 1] - v[i]);
  }

  void fail(Req<V>* q, int st) {
    char buf[512];
    ed_last_error(buf, sizeof(buf));
    q->status = st;
    q->err = buf;
    q->phase = PH_FAILED;
  }

  // ---- k > 1: the whole solve on a worker thread, on the request's stream,
  // with a sub-context of its own (private reduction scratch)
  int solve_k(Req<V>* q) {
    ED_TRY_CUDA(cudaSetDevice(ctx->device));
    q->sub.reset(new Ctx());
    ED_TRY(make_sub_ctx(ctx, q->sub.get()));
    q->sec.reset(new Sector());
    ED_TRY(build_sector(q->sub.get(), &q->model, q->n_up, q->n_dn, o.prec, q->sec.get()));
    ED_TRY(build_fast(q->sec.get()));
    const uint64_t n = q->sec->dim;
    const int kk = (int)std::min<uint64_t>((uint64_t)q->k, n);
    ed_trlan_opts to{};
    to.k = kk;
    to.tol = o.tol;
    to.max_basis = (int)std::min<uint64_t>((uint64_t)tr_basis(q->k), n);
    to.keep = 0;
    to.max_iter = o.max_iter;
    to.check_every = 4;
    to.seed = o.seed;
    to.v0 = nullptr;
    V* evecs = nullptr;
    ED_TRY(q->alloc(&evecs, (size_t)kk * n));
    std::vector<double> ev(std::max(kk, 1));
    ed_trlan_info info{};
    const int st = trlan_run(q->sec.get(), &to, ev.data(), evecs, &info, q->st);
    if (st != ED_OK && st != ED_ERR_NOT_CONVERGED) return st;
    q->Ek.assign(ev.begin(), ev.begin() + kk);
    q->E0 = ev[0];
    q->gs_iters = info.iters;
    if (q->want_G) {
      std::vector<ed_state> states(kk);
      for (int i = 0; i < kk; ++i) states[i] = ed_state{q->n_up, q->n_dn, ev[i], evecs + (size_t)i * n};
      q->G.assign(2 * (size_t)o.n_w, 0.0);
      ED_TRY(greens_cf_run(q->sub.get(), &q->model, o.prec, kk, states.data(), o.beta, o.n_w, nullptr, q->orbital,
                           q->spin, o.cf_depth, 1e-5, q->G.data(), nullptr, q->st));
    }
    ED_TRY_CUDA(cudaStreamSynchronize(q->st));
    return st;
  }

  void run_worker(Req<V>* q) {
    const int st = solve_k(q);
    if (st != ED_OK) {
      char buf[512];
      ed_last_error(buf, sizeof(buf));  // this thread's message
      q->status = st;
      q->err = st == ED_ERR_NOT_CONVERGED ? "thick-restart Lanczos did not converge within max_iter" : buf;
    }
    q->wdone = true;
  }

  // ---- a pack of small requests with the same k: their sectors' Lanczos runs
  // as one batched solve, then each request's Green's function; results are
  // written into the requests, phases are set by the server thread
  void run_pack(std::vector<Req<V>*> reqs) {
    int st = solve_pack(reqs);
    if (st != ED_OK) {
      char buf[512];
      ed_last_error(buf, sizeof(buf));
      for (Req<V>* q : reqs)
        if (q->status == ED_OK || q->status == ED_ERR_NOT_CONVERGED) {
          q->status = st;
          q->err = buf;
        }
    }
    pack_done = true;
  }

  int solve_pack(std::vector<Req<V>*>& reqs) {
    ED_TRY_CUDA(cudaSetDevice(ctx->device));
    Ctx sub;
    ED_TRY(make_sub_ctx(ctx, &sub));
    struct SubGuard {
      Ctx* c;
      ~SubGuard() { free_sub_ctx(c); }
    } sg{&sub};
    cudaStream_t st = nullptr;
    ED_TRY_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
      cudaStream_t s;
      ~StreamGuard() { cudaStreamDestroy(s); }
    } stg{st};
    const int n = (int)reqs.size(), k = reqs[0]->k;
    std::vector<const ed_model*> models(n);
    std::vector<int> nu(n), nd(n), it(n), conv(n);
    std::vector<void*> ritz(n, nullptr);
    std::vector<double> ev((size_t)n * k);
    struct Free {
      Ctx* c;
      std::vector<std::pair<void*, size_t>> v;
      ~Free() {
        for (auto& a : v) dev_free(c, a.first, a.second);
      }
    } fr{&sub, {}};
    for (int i = 0; i < n; ++i) {
      models[i] = &reqs[i]->model;
      nu[i] = reqs[i]->n_up;
      nd[i] = reqs[i]->n_dn;
      const size_t bytes = (size_t)std::min<uint64_t>((uint64_t)k, reqs[i]->dim) * reqs[i]->dim * sizeof(V);
      ED_TRY(dev_alloc(&sub, &ritz[i], bytes));
      fr.v.push_back({ritz[i], bytes});
    }
    ed_lanczos_opts lo{};
    lo.k = k;
    lo.tol = o.tol;
    lo.max_iter = std::min(o.max_iter, kPackIter);
    lo.check_every = 10;
    lo.seed = o.seed;
    lo.v0 = nullptr;
    lo.reorth = 1;
    const int bs = batch_solve_pack(&sub, o.prec, n, models.data(), nu.data(), nd.data(), &lo, kPackChunk,
                                    ev.data(), it.data(), conv.data(), ritz.data());
    if (bs != ED_OK && bs != ED_ERR_NOT_CONVERGED) return bs;
    for (int i = 0; i < n; ++i) {
      Req<V>* q = reqs[i];
      const int kk = (int)std::min<uint64_t>((uint64_t)k, q->dim);
      q->Ek.assign(ev.begin() + (size_t)i * k, ev.begin() + (size_t)i * k + kk);
      q->E0 = ev[(size_t)i * k];
      q->gs_iters = it[i];
      if (!conv[i]) {
        q->status = ED_ERR_NOT_CONVERGED;
        q->err = "packed Lanczos did not converge within its step limit";
      }
      if (q->want_G) {
        std::vector<ed_state> states(kk);
        for (int j = 0; j < kk; ++j)
          states[j] = ed_state{q->n_up, q->n_dn, q->Ek[j], static_cast<V*>(ritz[i]) + (size_t)j * q->dim};
        q->G.assign(2 * (size_t)o.n_w, 0.0);
        const int gs = greens_cf_run(&sub, &q->model, o.prec, kk, states.data(), o.beta, o.n_w, nullptr, q->orbital,
                                     q->spin, o.cf_depth, 1e-5, q->G.data(), nullptr, st);
        if (gs != ED_OK) {
          char buf[512];
          ed_last_error(buf, sizeof(buf));
          q->status = gs;
          q->err = buf;
        }
      }
    }
    ED_TRY_CUDA(cudaStreamSynchronize(st));
    return ED_OK;
  }

  int check_work(Req<V>* q) {
    if (!q->wdone) return ED_OK;
    q->worker.join();
    q->phase = (q->status == ED_OK || q->status == ED_ERR_NOT_CONVERGED) ? PH_DONE : PH_FAILED;
    return ED_OK;
  }

  // ---- per-request work, one call per server pass
  int admit(Req<V>* q) {
    cudaSetDevice(ctx->device);
    ED_TRY_CUDA(cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking));
    ED_TRY_CUDA(cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming));
    if (q->k > 1) {
      q->phase = PH_WORK;
      q->worker = std::thread([this, q] { run_worker(q); });
      return ED_OK;
    }
    ED_TRY_CUDA(cudaMallocHost(&q->h_pin, sizeof(double) * 4096));
    q->sec.reset(new Sector());
    ED_TRY(build_sector(ctx, &q->model, q->n_up, q->n_dn, o.prec, q->sec.get()));
    ED_TRY(build_fast(q->sec.get()));
    q->gs.reset(new Run3<V>());
    const int mmax = (int)std::min<uint64_t>((uint64_t)o.max_iter, q->sec->dim);
    ED_TRY(q->gs->init(q->sec.get(), ctx, q->st, std::max(mmax, 1), nullptr, o.seed, 1, 1e-13));
    const int ldS = mmax + 3;
    ED_TRY(q->alloc(&q->Sd, ldS));
    ED_TRY(q->alloc(&q->Sf, ldS));
    ED_TRY(q->alloc(&q->Sq, ldS));
    ED_TRY(q->alloc(&q->Sqf, ldS));
    ED_TRY(q->alloc(&q->theta, ED_MAX_K));
    ED_TRY(q->alloc(&q->resid, ED_MAX_K));
    ED_TRY(q->alloc(&q->twork, (size_t)6 * ldS));
    q->phase = PH_GS;
    return ED_OK;
  }

  int step_gs(Req<V>* q) {
    Run3<V>* r = q->gs.get();
    const int burst = 8;
    for (int b = 0; b < burst && r->launched < r->mmax; ++b) ED_TRY(r->launch_step());
    const bool at_check = (r->launched % 10 == 0) || r->launched >= r->mmax || q->sec->dim <= 64;
    if (!at_check) return ED_OK;
    // asynchronous convergence check: exhaustion flag, tridiagonal solve, residual
    const int m = r->launched;
    q->m_check = m;
    ED_TRY(tridiag(ctx, q->st, r->c, m, 1, 0.0, q->theta, q->Sd, q->Sf, r->mmax + 3, q->resid, q->twork));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin, q->theta, sizeof(double), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin + 1, q->Sd + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin + 2, r->c.beta + m, sizeof(double), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin + 3, r->c.exhausted, sizeof(int), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaEventRecord(q->ev, q->st));
    q->phase = PH_GS_CHECK;
    return ED_OK;
  }

  int check_gs(Req<V>* q) {
    cudaError_t e = cudaEventQuery(q->ev);
    if (e == cudaErrorNotReady) return ED_OK;
    ED_TRY_CUDA(e);
    Run3<V>* r = q->gs.get();
    int ex = -1;
    std::memcpy(&ex, q->h_pin + 3, sizeof(int));
    const double th = q->h_pin[0], last = q->h_pin[1], bm = q->h_pin[2];
    const bool exhausted = ex >= 0;
    const double res = exhausted ? 0.0 : std::fabs(bm * last);
    const bool conv = exhausted || res <= o.tol * std::max(1.0, std::fabs(th));
    if (!conv && r->launched < r->mmax) {
      q->phase = PH_GS;
      return ED_OK;
    }
    if (exhausted && ex < q->m_check) {
      // the check ran past the end of the Krylov space: redo it at the exhaustion step
      q->m_check = ex;
      ED_TRY(tridiag(ctx, q->st, r->c, ex, 1, 0.0, q->theta, q->Sd, q->Sf, r->mmax + 3, q->resid, q->twork));
      ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin, q->theta, sizeof(double), cudaMemcpyDeviceToHost, q->st));
      ED_TRY_CUDA(cudaStreamSynchronize(q->st));
    }
    q->m_final = q->m_check;
    q->E0 = q->h_pin[0];
    q->gs_iters = q->m_final;
    if (!conv) {
      q->status = ED_ERR_NOT_CONVERGED;
      q->err = "ground state not converged within max_iter";
    }
    if (!q->want_G) {
      q->phase = PH_DONE;
      return ED_OK;
    }
    // Ritz vector by regeneration: psi = sum_j S_j sigma_j q_j
    const int m = q->m_final;
    ED_TRY(q->alloc(&q->psi, q->sec->dim));
    ED_TRY_CUDA(cudaMemsetAsync(q->psi, 0, q->sec->dim * sizeof(V), q->st));
    k_scale_ritz<<<(m + 127) / 128, 128, 0, q->st>>>(q->Sd, r->c.sigma, m, 1, r->mmax + 3, q->Sq, q->Sqf);
    ED_TRY_CUDA(cudaMemcpyAsync(r->q(0), r->v0, q->sec->dim * sizeof(V), cudaMemcpyDeviceToDevice, q->st));
    q->vec_step = 0;
    q->phase = PH_VEC;
    return ED_OK;
  }

  int step_vec(Req<V>* q) {
    Run3<V>* r = q->gs.get();
    const uint64_t n = q->sec->dim;
    uint32_t vg = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 16);
    if (!vg) vg = 1;
    const int burst = 8;
    for (int b = 0; b < burst && q->vec_step < q->m_final; ++b) {
      const int jj = q->vec_step;
      k_ritz<V, 8><<<vg, 256, 0, q->st>>>(r->q(jj), n, 1, q->Sq + jj, q->Sqf + jj, r->mmax + 3, 0, 1, q->psi, n, 1);
      if (jj + 1 < q->m_final) {
        ED_TRY(apply_h(q->sec.get(), r->q(jj), r->Y, q->st));
        k_lz_step<V><<<r->sgrid, kRedThreads, 0, q->st>>>(r->Y, r->q(jj), jj > 0 ? r->q(jj - 1) : nullptr,
                                                          r->q(jj + 1), n, r->c, jj, nullptr);
      }
      ED_LAUNCH_CHECK();
      ++q->vec_step;
    }
    if (q->vec_step < q->m_final) return ED_OK;
    // unit norm: a ghost copy of the converged ground state (loss of
    // orthogonality, early with float vectors) leaves sum_j S_j v_j unnormalised
    k_dot<V><<<r->sgrid, kRedThreads, 0, q->st>>>(q->psi, q->psi, n, r->partial);
    k_finish<<<1, kRedThreads, 0, q->st>>>(r->partial, (int)r->sgrid, OP_NORM_INV, 0, r->c, 0.0);
    k_rescale<V><<<vg, 256, 0, q->st>>>(q->psi, n, r->c, 0);
    ED_LAUNCH_CHECK();
    ED_TRY_CUDA(cudaStreamSynchronize(q->st));  // r->c is freed with the ground-state run
    q->gs.reset();  // ground-state buffers are no longer needed
    ED_TRY(q->alloc(&q->dG, o.n_w));
    ED_TRY(q->alloc(&q->dE, 1));
    ED_TRY(q->alloc(&q->dab, 2 * (size_t)o.cf_depth));
    ED_TRY_CUDA(cudaMemsetAsync(q->dG, 0, sizeof(double2) * o.n_w, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->dE, &q->E0, sizeof(double), cudaMemcpyHostToDevice, q->st));
    ED_TRY_CUDA(cudaStreamSynchronize(q->st));
    q->cf_part = 0;
    return start_cf(q);
  }

  int start_cf(Req<V>* q) {
    while (q->cf_part < 2) {
      const bool dag = q->cf_part == 0;
      const int tu = q->n_up + (q->spin == ED_SPIN_UP ? (dag ? 1 : -1) : 0);
      const int td = q->n_dn + (q->spin == ED_SPIN_DN ? (dag ? 1 : -1) : 0);
      const int ns = q->model.n_s;
      if (tu < 0 || tu > ns || td < 0 || td > ns) {
        ++q->cf_part;
        continue;
      }
      if (q->sec_cf) free_sector(q->sec_cf.get());
      q->sec_cf.reset(new Sector());
      ED_TRY(build_sector(ctx, &q->model, tu, td, o.prec, q->sec_cf.get()));
      ED_TRY(build_fast(q->sec_cf.get()));
      V* phi = nullptr;
      ED_TRY(dev_alloc(ctx, reinterpret_cast<void**>(&phi), q->sec_cf->dim * sizeof(V)));
      int st = apply_cop(q->sec.get(), q->sec_cf.get(), q->orbital, q->spin, dag, q->psi, phi, q->st);
      if (st == ED_OK) {
        q->cf.reset(new Run3<V>());
        st = q->cf->init(q->sec_cf.get(), ctx, q->st, o.cf_depth, phi, 0, 1, 1e-12);
      }
      cudaStreamSynchronize(q->st);
      dev_free(ctx, phi, q->sec_cf->dim * sizeof(V));
      if (st != ED_OK) return st;
      q->phase = PH_CF;
      return ED_OK;
    }
    // both parts done (or empty): copy G to the host
    q->G.assign(2 * (size_t)o.n_w, 0.0);
    ED_TRY_CUDA(cudaMemcpyAsync(q->G.data(), q->dG, sizeof(double2) * o.n_w, cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaEventRecord(q->ev, q->st));
    q->phase = PH_EVAL_WAIT;
    return ED_OK;
  }

  int step_cf(Req<V>* q) {
    Run3<V>* r = q->cf.get();
    const int burst = 8;
    for (int b = 0; b < burst && r->launched < r->mmax; ++b) ED_TRY(r->launch_step());
    if (r->launched < r->mmax) return ED_OK;
    // coefficients to the pinned staging buffer
    const int L = r->mmax;
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin, r->c.alpha, sizeof(double) * L, cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin + 1024, r->c.beta, sizeof(double) * (L + 1), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin + 2048, r->c.out, sizeof(double), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaMemcpyAsync(q->h_pin + 2049, r->c.exhausted, sizeof(int), cudaMemcpyDeviceToHost, q->st));
    ED_TRY_CUDA(cudaEventRecord(q->ev, q->st));
    q->phase = PH_CF_WAIT;
    return ED_OK;
  }

  int finish_cf(Req<V>* q) {
    cudaError_t e = cudaEventQuery(q->ev);
    if (e == cudaErrorNotReady) return ED_OK;
    ED_TRY_CUDA(e);
    const int depth = q->cf->mmax;
    int ex = -1;
    std::memcpy(&ex, q->h_pin + 2049, sizeof(int));
    const double norm = q->h_pin[2048];
    int len = (ex >= 0 && ex < depth) ? ex : depth;
    if (norm == 0.0) len = 0;
    std::vector<double> ab(2 * (size_t)depth, 0.0);
    for (int i = 0; i < len; ++i) {
      ab[i] = q->h_pin[i];
      ab[depth + i] = i > 0 ? q->h_pin[1024 + i] : 0.0;
    }
    if (len > 0) {
      ED_TRY_CUDA(cudaMemcpyAsync(q->dab, ab.data(), sizeof(double) * 2 * depth, cudaMemcpyHostToDevice, q->st));
      ED_TRY(greens_accumulate(q->dG, o.n_w, o.beta, q->dab, q->dab + depth, len, norm * norm, q->dE, 1, 0,
                               q->cf_part == 0 ? 1 : -1, q->st));
      ED_TRY_CUDA(cudaStreamSynchronize(q->st));  // ab is reused by the next part
    }
    q->cf.reset();
    ++q->cf_part;
    return start_cf(q);
  }

  int check_eval(Req<V>* q) {
    cudaError_t e = cudaEventQuery(q->ev);
    if (e == cudaErrorNotReady) return ED_OK;
    ED_TRY_CUDA(e);
    q->phase = PH_DONE;
    return ED_OK;
  }

  int advance(Req<V>* q) {
    switch (q->phase) {
      case PH_GS: return step_gs(q);
      case PH_GS_CHECK: return check_gs(q);
      case PH_VEC: return step_vec(q);
      case PH_CF: return step_cf(q);
      case PH_CF_WAIT: return finish_cf(q);
      case PH_EVAL_WAIT: return check_eval(q);
      case PH_WORK: return check_work(q);
      default: return ED_OK;
    }
  }

  void loop() {
    cudaSetDevice(ctx->device);
    while (!stop) {
      // a finished pack: its requests are done (or failed)
      if (pack_running && pack_done) {
        pack_th.join();
        pack_running = false;
        for (Req<V>* q : pack_reqs)
          q->phase = (q->status == ED_OK || q->status == ED_ERR_NOT_CONVERGED) ? PH_DONE : PH_FAILED;
        pack_reqs.clear();
      }
      // a new pack: the queued small requests with the first one's k, while their footprint fits
      if (!pack_running) {
        std::lock_guard<std::mutex> lk(mu);
        if (!pack_q.empty()) {
          const int k = pack_q.front()->k;
          std::deque<std::unique_ptr<Req<V>>> rest;
          const double t_now = now_ms();
          while (!pack_q.empty()) {
            std::unique_ptr<Req<V>> q = std::move(pack_q.front());
            pack_q.pop_front();
            const bool fits = !o.hbm_budget || in_flight_bytes + q->footprint <= o.hbm_budget ||
                              (active.empty() && pack_reqs.empty());
            if (q->k != k || (int)pack_reqs.size() >= kMaxPack || !fits) {
              rest.push_back(std::move(q));
              continue;
            }
            in_flight_bytes += q->footprint;
            q->t_admit = t_now;
            q->phase = PH_PACK;
            pack_reqs.push_back(q.get());
            active.push_back(std::move(q));
          }
          pack_q = std::move(rest);
          if (!pack_reqs.empty()) {
            max_active_seen = std::max(max_active_seen, (int)active.size());
            pack_done = false;
            pack_running = true;
            pack_th = std::thread([this, reqs = pack_reqs] { run_pack(reqs); });
          }
        }
      }
      // admissions, first come first served, by HBM footprint and slot count
      for (;;) {
        std::unique_ptr<Req<V>> q;
        {
          std::lock_guard<std::mutex> lk(mu);
          if (queue.empty()) break;
          if (queue.front()->packed) {  // small requests wait for the next pack
            pack_q.push_back(std::move(queue.front()));
            queue.pop_front();
            continue;
          }
          const size_t need = queue.front()->footprint;
          int slots = 0;  // packed requests take no slot
          for (auto& a : active) slots += a->packed ? 0 : 1;
          if (slots >= o.max_active) break;
          if (o.hbm_budget && in_flight_bytes + need > o.hbm_budget && !active.empty()) break;
          q = std::move(queue.front());
          queue.pop_front();
          in_flight_bytes += q->footprint;
        }
        q->t_admit = now_ms();
        int st = admit(q.get());
        if (st != ED_OK) fail(q.get(), st);
        std::lock_guard<std::mutex> lk(mu);
        active.push_back(std::move(q));
        max_active_seen = std::max(max_active_seen, (int)active.size());
      }
      // nothing to drive on this thread when every active request waits on a worker
      bool idle = true;
      for (auto& q : active) {
        if (q->phase == PH_DONE || q->phase == PH_FAILED) continue;
        if (q->phase != PH_WORK && q->phase != PH_PACK) idle = false;
        int st = advance(q.get());
        if (st != ED_OK) fail(q.get(), st);
      }
      // retire finished requests
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < active.size();) {
          Req<V>* q = active[i].get();
          if (q->phase == PH_DONE || q->phase == PH_FAILED) {
            if (q->st) cudaStreamSynchronize(q->st);
            q->t_done = now_ms();
            in_flight_bytes -= std::min(in_flight_bytes, q->footprint);
            if (q->phase == PH_DONE && q->status == ED_OK) ++n_done;
            else ++n_failed;
            lat_ms.push_back(q->t_done - q->t_submit);
            wait_ms.push_back(q->t_admit - q->t_submit);
            q->release();
            finished[q->ticket] = std::move(active[i]);
            active.erase(active.begin() + i);
          } else {
            ++i;
          }
        }
      }
      if (idle) {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait_for(lk, std::chrono::microseconds(200), [this] { return stop || !queue.empty(); });
      }
    }
  }
};

}  // namespace

}  // namespace ed

using namespace ed;

struct ed_server {
  std::unique_ptr<ServerBase> s;
};

extern "C" int ed_server_create(ed_ctx* ctx, const ed_server_opts* opts, ed_server** out) {
  if (!ctx || !opts || !out) ED_INVALID("NULL argument");
  *out = nullptr;
  ed_server_opts o = *opts;
  if (o.max_active < 1) ED_INVALID("max_active must be >= 1");
  if (o.max_iter < 1 || !(o.tol > 0.0)) ED_INVALID("bad max_iter / tol");
  if (o.cf_depth < 1 || o.cf_depth > 1000) ED_INVALID("cf_depth outside 1..1000");
  if (o.n_w < 1 || !(o.beta > 0.0)) ED_INVALID("bad n_w / beta");
  if (o.prec != ED_PREC_FP64 && o.prec != ED_PREC_DF64 && o.prec != ED_PREC_FP32) ED_INVALID("unknown precision");
  Ctx* c = ctx_of(ctx);
  std::unique_ptr<ed_server> h(new ed_server());
  try {
    switch (o.prec) {
      case ED_PREC_FP64: h->s.reset(new Server<double>(c, o)); break;
      case ED_PREC_DF64: h->s.reset(new Server<float2>(c, o)); break;
      default: h->s.reset(new Server<float>(c, o));
    }
  } catch (...) {
    ED_INVALID("could not start the server thread");
  }
  *out = h.release();
  return ED_OK;
}

extern "C" int ed_server_destroy(ed_server* s) {
  if (!s) return ED_OK;
  delete s;
  return ED_OK;
}

extern "C" int ed_submit(ed_server* s, const ed_request* r, uint64_t* ticket) {
  if (!s || !r || !r->model || !ticket) ED_INVALID("NULL argument");
  try {
    return s->s->submit(r, ticket);
  } catch (...) {
    set_error("submit failed");
    return ED_ERR_OOM;
  }
}

extern "C" int ed_poll(ed_server* s, uint64_t ticket, ed_result* res, double* G, int* done) {
  if (!s || !done) ED_INVALID("NULL argument");
  return s->s->poll(ticket, res, G, done);
}

extern "C" int ed_server_get_stats(ed_server* s, ed_server_stats* st) {
  if (!s || !st) ED_INVALID("NULL argument");
  return s->s->stats(st);
}
