// Lanczos recurrence around the sector H*v (Sec. 3: iterative eigensolvers
// built on repeated multiplication of H by a trial vector), entirely on the
// device:
//   w = H v_j;  alpha_j = <v_j, w>;  w -= alpha_j v_j + beta_j v_{j-1};
//   [full reorthogonalisation: twice  h = V^T w, w -= V h  (CGS2)]
//   beta_{j+1} = |w|;  v_{j+1} = w / beta_{j+1}.
// Dot products and norms are accumulated in double (FP64 vectors) or in
// double-float (DF64 and FP32 vectors) and reduced to double; alpha, beta and
// the tridiagonal eigenproblem are FP64.  The tridiagonal eigensolver is
// Sturm-sequence multisection for the eigenvalues plus inverse iteration
// (tridiagonal Gaussian elimination with partial pivoting) for the vectors.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lanczos_kernels.h"

namespace ed {

size_t elem_bytes(int prec) {
  switch (prec) {
    case ED_PREC_FP64: return 8;
    case ED_PREC_DF64: return 8;
    case ED_PREC_FP32: return 4;
  }
  return 0;
}

namespace {
// Three-vector recurrence on unnormalised vectors (v_j = sigma_j q_j), two
// large kernels per step: H q_j fused with <q_j, H q_j>, then the update fused
// with |q_{j+1}|^2.  The coefficients stay on the device.
template <class V>
struct Rec3 {
  Sector* s;
  Work<V>* W;
  V* Q[3];  // q_{j-1}, q_j, q_{j+1} rotate through these
  V* Y;     // H q_j
  uint32_t sgrid;
  V* q(int j) { return Q[((j % 3) + 3) % 3]; }

  int apply_dot(const V* x, V* y, int* np) {
    if (s->fast.ok) return apply_fast(s, x, y, W->st, W->partial, np);
    ED_TRY(apply_h(s, x, y, W->st));
    k_dot<V><<<W->grid, kRedThreads, 0, W->st>>>(x, y, W->n, W->partial);
    ED_LAUNCH_CHECK();
    *np = (int)W->grid;
    return ED_OK;
  }
  int init() {  // q_0 already in Q[0]
    return dot_to(*W, (const V*)q(0), (const V*)q(0), OP_SIGMA0, 0);
  }
  int step(int j, double thr, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
    int np = 0;
    if (e0) ED_TRY_CUDA(cudaEventRecord(e0, W->st));
    ED_TRY(apply_dot(q(j), Y, &np));
    if (e1) ED_TRY_CUDA(cudaEventRecord(e1, W->st));
    k_finish<<<1, kRedThreads, 0, W->st>>>(W->partial, np, OP_ALPHA_Q, j, W->c, 0.0);
    k_lz_step<V><<<sgrid, kRedThreads, 0, W->st>>>(Y, q(j), j > 0 ? q(j - 1) : nullptr, q(j + 1), W->n, W->c, j,
                                                   W->partial);
    k_finish<<<1, kRedThreads, 0, W->st>>>(W->partial, (int)sgrid, OP_BETA_Q, j + 1, W->c, thr);
    ED_LAUNCH_CHECK();
    return ED_OK;
  }
  // Regenerate q_{j+1} from q_j, q_{j-1} with the stored coefficients.
  int regen(int j) {
    ED_TRY(apply_h(s, q(j), Y, W->st));
    k_lz_step<V><<<sgrid, kRedThreads, 0, W->st>>>(Y, q(j), j > 0 ? q(j - 1) : nullptr, q(j + 1), W->n, W->c, j,
                                                   nullptr);
    ED_LAUNCH_CHECK();
    return ED_OK;
  }
};

template <class V>
int coeffs_impl(Sector* s, const void* phi, int depth, double* n2, double* a, double* b, int* L,
                cudaStream_t st) {
  Ctx* ctx = s->ctx;
  const uint64_t n = s->dim;
  size_t eb = sizeof(V);
  DevBuf vb, cb;
  ED_TRY(vb.alloc(ctx, 4 * n * eb));
  ED_TRY(cb.alloc(ctx, coef_bytes(depth, 1)));
  V* vecs = static_cast<V*>(vb.p);
  Carve cv{static_cast<char*>(cb.p)};
  Coefs c = carve_coefs(cv, depth);
  Work<V> W;
  W.ctx = ctx;
  W.st = st;
  W.n = n;
  W.grid = (uint32_t)std::min<uint64_t>((n + kRedThreads - 1) / kRedThreads, (uint64_t)ctx->num_sms * 8);
  if (W.grid == 0) W.grid = 1;
  W.partial = ctx->d_red;
  W.c = c;
  Rec3<V> R{s, &W, {vecs, vecs + n, vecs + 2 * n}, vecs + 3 * n, W.grid};
  k_init_coefs<<<1, 256, 0, st>>>(c, depth + 2);
  ED_TRY_CUDA(cudaMemcpyAsync(R.q(0), phi, n * eb, cudaMemcpyDeviceToDevice, st));
  ED_TRY(R.init());
  const double thr = 1e-12;
  for (int j = 0; j < depth; ++j) ED_TRY(R.step(j, thr));
  std::vector<double> hb(depth + 1), ha(depth);
  double norm = 0.0;
  int ex = -1;
  ED_TRY_CUDA(cudaMemcpyAsync(ha.data(), c.alpha, depth * sizeof(double), cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaMemcpyAsync(hb.data(), c.beta, (depth + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaMemcpyAsync(&norm, c.out, sizeof(double), cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaMemcpyAsync(&ex, c.exhausted, sizeof(int), cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  *n2 = norm * norm;
  int len = (ex >= 0 && ex < depth) ? ex : depth;
  if (norm == 0.0) len = 0;
  *L = len;
  for (int i = 0; i < depth; ++i) {
    a[i] = (i < len) ? ha[i] : 0.0;
    b[i] = (i < len && i > 0) ? hb[i] : 0.0;
  }
  return ED_OK;
}

// Lanczos without reorthogonalisation: three resident vectors, eigenvalues from
// the tridiagonal matrix, Ritz vectors by a second pass that regenerates the
// same q_j with the stored coefficients.
template <class V>
int lanczos3_impl(Sector* s, const ed_lanczos_opts* o, double* evals, void* evecs, ed_lanczos_info* info,
                  cudaStream_t st) {
  auto t_start = std::chrono::steady_clock::now();
  Ctx* ctx = s->ctx;
  const uint64_t n = s->dim;
  const int k = o->k;
  int mmax = (int)std::min<uint64_t>((uint64_t)o->max_iter, n);
  if (mmax < 1) mmax = 1;
  const int check_every = std::max(1, o->check_every);
  const int kk = std::min<int>(k, (int)n);
  size_t eb = sizeof(V);
  DevBuf vb, cb, v0b;
  ED_TRY(vb.alloc(ctx, 4 * n * eb));
  ED_TRY(v0b.alloc(ctx, n * eb));
  ED_TRY(cb.alloc(ctx, coef_bytes(mmax, std::max(kk, 1))));
  V* vecs = static_cast<V*>(vb.p);
  Carve cv{static_cast<char*>(cb.p)};
  Coefs c = carve_coefs(cv, mmax);
  int ldS = mmax + 1;
  double* theta = cv.take<double>(ED_MAX_K);
  double* resid = cv.take<double>(ED_MAX_K);
  double* Sd = cv.take<double>((size_t)ldS * std::max(kk, 1));
  float2* Sf = cv.take<float2>((size_t)ldS * std::max(kk, 1));
  double* Sq = cv.take<double>((size_t)ldS * std::max(kk, 1));
  float2* Sqf = cv.take<float2>((size_t)ldS * std::max(kk, 1));
  double* twork = cv.take<double>((size_t)6 * ldS * std::max(kk, 1));
  Work<V> W;
  W.ctx = ctx;
  W.st = st;
  W.n = n;
  W.grid = (uint32_t)std::min<uint64_t>((n + kRedThreads - 1) / kRedThreads, (uint64_t)ctx->num_sms * 8);
  if (W.grid == 0) W.grid = 1;
  W.partial = ctx->d_red;
  W.c = c;
  uint32_t vgrid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 16);
  if (vgrid == 0) vgrid = 1;
  Rec3<V> R{s, &W, {vecs, vecs + n, vecs + 2 * n}, vecs + 3 * n, W.grid};
  k_init_coefs<<<1, 256, 0, st>>>(c, mmax + 2);
  if (o->v0) {
    ED_TRY_CUDA(cudaMemcpyAsync(R.q(0), o->v0, n * eb, cudaMemcpyDeviceToDevice, st));
  } else {
    k_random<V><<<vgrid, 256, 0, st>>>(R.q(0), n, o->seed);
  }
  ED_TRY_CUDA(cudaMemcpyAsync(v0b.p, R.q(0), n * eb, cudaMemcpyDeviceToDevice, st));
  ED_TRY(R.init());
  std::vector<double> h_theta(ED_MAX_K), h_res(ED_MAX_K);
  int m = 0, n_conv = 0, status = ED_OK;
  const double thr = 1e-13;
  // one event pair per step times the H*v launches of the recurrence
  std::vector<cudaEvent_t> evs(2 * (size_t)mmax);
  for (auto& e : evs) ED_TRY_CUDA(cudaEventCreate(&e));
  struct EvGuard {
    std::vector<cudaEvent_t>* v;
    ~EvGuard() {
      for (auto e : *v) cudaEventDestroy(e);
    }
  } evguard{&evs};
  int n_steps = 0;
  for (int j = 0; j < mmax; ++j) {
    ED_TRY(R.step(j, thr, evs[2 * j], evs[2 * j + 1]));
    n_steps = j + 1;
    m = j + 1;
    bool check = ((m % check_every) == 0) || (m == mmax) || (n <= 4096);
    if (!check) continue;
    int ex = -1;
    ED_TRY_CUDA(cudaMemcpyAsync(ctx->h_red, c.exhausted, sizeof(int), cudaMemcpyDeviceToHost, st));
    ED_TRY_CUDA(cudaStreamSynchronize(st));
    std::memcpy(&ex, ctx->h_red, sizeof(int));
    bool exhausted = ex >= 0;
    if (exhausted) m = ex;
    int kc = std::min(kk, m);
    ED_TRY(tridiag(ctx, st, c, m, kc, 0.0, theta, Sd, Sf, ldS, resid, twork));
    std::vector<double> last(kc);
    double bm = 0.0;
    ED_TRY_CUDA(cudaMemcpyAsync(&bm, c.beta + m, sizeof(double), cudaMemcpyDeviceToHost, st));
    ED_TRY_CUDA(cudaMemcpyAsync(h_theta.data(), theta, kc * sizeof(double), cudaMemcpyDeviceToHost, st));
    for (int i = 0; i < kc; ++i)
      ED_TRY_CUDA(cudaMemcpyAsync(&last[i], Sd + (size_t)i * ldS + m - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    ED_TRY_CUDA(cudaStreamSynchronize(st));
    if (exhausted) bm = 0.0;
    n_conv = 0;
    for (int i = 0; i < kc; ++i) {
      h_res[i] = std::fabs(bm * last[i]);
      if (h_res[i] <= o->tol * std::max(1.0, std::fabs(h_theta[i])) && n_conv == i) ++n_conv;
    }
    if (exhausted || (kc >= kk && n_conv >= kk)) break;
    if (m >= mmax) status = ED_ERR_NOT_CONVERGED;
  }
  if (m >= mmax && n_conv < kk) status = ED_ERR_NOT_CONVERGED;
  int kc = std::min(kk, m);
  for (int i = 0; i < kc; ++i) evals[i] = h_theta[i];
  for (int i = kc; i < k; ++i) evals[i] = NAN;
  if (info) {
    info->iters = m;
    info->n_converged = std::min(n_conv, kc);
    for (int i = 0; i < ED_MAX_K; ++i) info->residual[i] = (i < kc) ? h_res[i] : 0.0;
  }
  if (evecs && kc > 0) {
    ED_TRY(tridiag(ctx, st, c, m, kc, 0.0, theta, Sd, Sf, ldS, resid, twork));
    k_scale_ritz<<<(m * kc + 127) / 128, 128, 0, st>>>(Sd, c.sigma, m, kc, ldS, Sq, Sqf);
    V* out = static_cast<V*>(evecs);
    ED_TRY_CUDA(cudaMemsetAsync(out, 0, (size_t)kc * n * eb, st));
    ED_TRY_CUDA(cudaMemcpyAsync(R.q(0), v0b.p, n * eb, cudaMemcpyDeviceToDevice, st));
    for (int jj = 0; jj < m; ++jj) {
      for (int i0 = 0; i0 < kc; i0 += 8)
        k_ritz<V, 8><<<vgrid, 256, 0, st>>>(R.q(jj), n, 1, Sq + jj, Sqf + jj, ldS, i0, std::min(8, kc - i0), out, n, 1);
      if (jj + 1 == m) break;
      ED_TRY(R.regen(jj));
    }
    ED_LAUNCH_CHECK();
    // unit norm (a ghost copy of a converged value leaves sum_j S_j v_j unnormalised)
    for (int i = 0; i < kc; ++i) {
      ED_TRY(dot_to(W, (const V*)(out + (size_t)i * n), (const V*)(out + (size_t)i * n), OP_NORM_INV, 0));
      k_rescale<V><<<vgrid, 256, 0, st>>>(out + (size_t)i * n, n, c, 0);
    }
    ED_LAUNCH_CHECK();
  }
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  if (info) {
    double apply_ms = 0.0;
    for (int q = 0; q < n_steps; ++q) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, evs[2 * q], evs[2 * q + 1]) == cudaSuccess) apply_ms += ms;
    }
    info->apply_ms = apply_ms;
    info->total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  }
  if (status != ED_OK) set_error("Lanczos did not converge in %d steps", mmax);
  return status;
}

}  // namespace

int dot_async(Ctx* c, const void* x, const void* y, uint64_t n, int prec, double* d_out, cudaStream_t st) {
  uint32_t grid = (uint32_t)std::min<uint64_t>((n + kRedThreads - 1) / kRedThreads, (uint64_t)c->num_sms * 8);
  if (grid == 0) grid = 1;
  Coefs cf{};
  cf.out = d_out;
  switch (prec) {
    case ED_PREC_FP64:
      k_dot<double><<<grid, kRedThreads, 0, st>>>((const double*)x, (const double*)y, n, c->d_red);
      break;
    case ED_PREC_DF64:
      k_dot<float2><<<grid, kRedThreads, 0, st>>>((const float2*)x, (const float2*)y, n, c->d_red);
      break;
    case ED_PREC_FP32:
      k_dot<float><<<grid, kRedThreads, 0, st>>>((const float*)x, (const float*)y, n, c->d_red);
      break;
    default: ED_INVALID("unknown precision %d", prec);
  }
  k_finish<<<1, kRedThreads, 0, st>>>(c->d_red, (int)grid, OP_SUM, 0, cf, 0.0);
  ED_LAUNCH_CHECK();
  return ED_OK;
}

int lanczos_run(Sector* s, const ed_lanczos_opts* o, double* evals, void* evecs, ed_lanczos_info* info,
                cudaStream_t st) {
  if (!o->reorth) {
    switch (s->prec) {
      case ED_PREC_FP64: return lanczos3_impl<double>(s, o, evals, evecs, info, st);
      case ED_PREC_DF64: return lanczos3_impl<float2>(s, o, evals, evecs, info, st);
      case ED_PREC_FP32: return lanczos3_impl<float>(s, o, evals, evecs, info, st);
    }
  }
  switch (s->prec) {
    case ED_PREC_FP64: return lanczos_impl<double>(s, o, evals, evecs, info, st);
    case ED_PREC_DF64: return lanczos_impl<float2>(s, o, evals, evecs, info, st);
    case ED_PREC_FP32: return lanczos_impl<float>(s, o, evals, evecs, info, st);
  }
  ED_INVALID("unknown precision");
}

int lanczos_coeffs(Sector* s, const void* phi, int depth, double* n2, double* a, double* b, int* L,
                   cudaStream_t st) {
  switch (s->prec) {
    case ED_PREC_FP64: return coeffs_impl<double>(s, phi, depth, n2, a, b, L, st);
    case ED_PREC_DF64: return coeffs_impl<float2>(s, phi, depth, n2, a, b, L, st);
    case ED_PREC_FP32: return coeffs_impl<float>(s, phi, depth, n2, a, b, L, st);
  }
  ED_INVALID("unknown precision");
}

}  // namespace ed
