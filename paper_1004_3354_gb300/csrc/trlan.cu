// Thick-restart Lanczos (Wu & Simon, SIAM J. Matrix Anal. Appl. 22, 2000) for
// the k lowest eigenpairs of a sector Hamiltonian with a Krylov basis of at
// most m vectors.
//
// The paper's solver is the implicitly restarted Arnoldi method (abstract;
// Sec. 3).  For a symmetric H, an implicit restart whose shifts are the
// unwanted Ritz values keeps the span of the wanted Ritz vectors and the
// residual direction; a thick restart keeps that span explicitly:
//
//   after m steps   H V_m = V_m H_m + beta_m v_m e_m^T,   H_m Y = Y Theta,
//   keep u_i = V_m y_i (i < l) and v_l = v_m; the projected matrix becomes
//     [[diag(theta_0 .. theta_{l-1}), s], [s^T, alpha_l, beta_{l+1}], ...]
//   with s_i = beta_m Y[m-1][i] (an arrow on a tridiagonal), and the recurrence
//   continues from v_l with full CGS2 reorthogonalisation against every
//   basis vector (which also removes the s_i u_i components of H v_l).
//
// The projected eigenproblem (dense, symmetric, at most ED_MAX_BASIS rows) is
// solved on the device by cyclic Jacobi in one block (round-robin pairs, all
// disjoint rotations of a round at once); the basis rotation V_m Y is k_ritz.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lanczos_kernels.h"

namespace ed {

namespace {

constexpr int kMaxBasis = ED_MAX_BASIS;
constexpr int kJacThreads = 512;

// Eigen-decomposition of the m x m symmetric matrix Ain (row-major, leading
// dimension lda): theta ascending, eigenvector i in S[i * ldS + r] (and its
// double-float split in Sf).  Y is m * m doubles of device scratch.
__global__ void __launch_bounds__(kJacThreads) k_sym_jacobi(const double* __restrict__ Ain, int m, int lda,
                                                            double* __restrict__ theta, double* __restrict__ S,
                                                            float2* __restrict__ Sf, int ldS, double* __restrict__ Y,
                                                            int* __restrict__ sweeps) {
  extern __shared__ double A[];  // m x m, row stride m
  __shared__ double cs[kMaxBasis / 2], sn[kMaxBasis / 2];
  __shared__ int pp[kMaxBasis / 2], qq[kMaxBasis / 2];
  __shared__ double red[kJacThreads / 32];
  __shared__ int order[kMaxBasis];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m * m; i += nt) {
    A[i] = Ain[(size_t)(i / m) * lda + i % m];
    Y[i] = (i / m == i % m) ? 1.0 : 0.0;
  }
  __syncthreads();
  auto block_sum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t += red[w];
    __syncthreads();
    return t;
  };
  double fro = 0.0;
  for (int i = tid; i < m * m; i += nt) fro += A[i] * A[i];
  fro = block_sum(fro);
  const int mp = m + (m & 1);  // players; index m is a dummy when m is odd
  const int np = mp / 2;
  int sweep = 0;
  for (; sweep < 60 && m > 1; ++sweep) {
    double off = 0.0;
    for (int i = tid; i < m * m; i += nt)
      if (i / m != i % m) off += A[i] * A[i];
    off = block_sum(off);
    if (!(off > 1e-32 * fro)) break;
    for (int r = 0; r < mp - 1; ++r) {
      for (int i = tid; i < np; i += nt) {
        const int a = (i == 0) ? 0 : ((i - 1 + r) % (mp - 1)) + 1;
        const int b = ((mp - 2 - i + r) % (mp - 1)) + 1;
        const int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p * m + q];
          if (apq != 0.0) {
            const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pp[i] = p;
        qq[i] = q;
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      // A <- J^T A (rows p, q of each pair)
      for (int idx = tid; idx < np * m; idx += nt) {
        const int i = idx / m, col = idx % m, p = pp[i], q = qq[i];
        if (q >= m) continue;
        const double c = cs[i], s = sn[i], ap = A[p * m + col], aq = A[q * m + col];
        A[p * m + col] = c * ap - s * aq;
        A[q * m + col] = s * ap + c * aq;
      }
      __syncthreads();
      // A <- A J (columns p, q) and the eigenvector matrix (Y holds its columns as rows)
      for (int idx = tid; idx < np * m; idx += nt) {
        const int i = idx / m, row = idx % m, p = pp[i], q = qq[i];
        if (q >= m) continue;
        const double c = cs[i], s = sn[i];
        const double ap = A[row * m + p], aq = A[row * m + q];
        A[row * m + p] = c * ap - s * aq;
        A[row * m + q] = s * ap + c * aq;
        const double yp = Y[p * m + row], yq = Y[q * m + row];
        Y[p * m + row] = c * yp - s * yq;
        Y[q * m + row] = s * yp + c * yq;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 1; i < m; ++i) {  // insertion sort by eigenvalue
      const int v = order[i];
      const double key = A[v * m + v];
      int j = i - 1;
      while (j >= 0 && A[order[j] * m + order[j]] > key) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = v;
    }
    if (sweeps) *sweeps = sweep;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) theta[i] = A[order[i] * m + order[i]];
  for (int idx = tid; idx < m * m; idx += nt) {
    const int i = idx / m, r = idx % m;
    const double v = Y[order[i] * m + r];
    S[(size_t)i * ldS + r] = v;
    Sf[(size_t)i * ldS + r] = df_from_double(v);
  }
}

// Projected matrix of the current basis (size rows): the kept Ritz values and
// their couplings s to basis vector l, then the Lanczos tridiagonal from l on.
__global__ void k_tr_project(double* __restrict__ Hp, int ld, int size, int l, const double* __restrict__ th,
                             const double* __restrict__ sv, Coefs c) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < size * size; idx += gridDim.x * blockDim.x) {
    const int i = idx / size, j = idx % size;
    double v = 0.0;
    if (i == j) v = (i < l) ? th[i] : c.alpha[i];
    else if (i < l && j == l) v = sv[i];
    else if (j < l && i == l) v = sv[j];
    else if (i >= l && j == i + 1) v = c.beta[j];
    else if (j >= l && i == j + 1) v = c.beta[i];
    Hp[(size_t)i * ld + j] = v;
  }
}

// After a restart with l kept vectors: theta and s_i = beta_m S[i][m-1].
__global__ void k_tr_keep(const double* __restrict__ theta, const double* __restrict__ S, int ldS, int m, int l,
                          Coefs c, double* __restrict__ th, double* __restrict__ sv) {
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    th[i] = theta[i];
    sv[i] = c.beta[m] * S[(size_t)i * ldS + m - 1];
  }
}

int jacobi(cudaStream_t st, const double* Hp, int m, int ld, double* theta, double* S, float2* Sf, int ldS,
           double* Y) {
  const size_t smem = (size_t)m * m * sizeof(double);
  // one cap for every size (kMaxBasis^2 doubles): concurrent solves of different
  // basis sizes set the same value
  ED_TRY_CUDA(cudaFuncSetAttribute(k_sym_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)((size_t)kMaxBasis * kMaxBasis * sizeof(double))));
  k_sym_jacobi<<<1, kJacThreads, smem, st>>>(Hp, m, ld, theta, S, Sf, ldS, Y, nullptr);
  ED_LAUNCH_CHECK();
  return ED_OK;
}

template <class V>
int trlan_impl(Sector* s, const ed_trlan_opts* o, double* evals, void* evecs, ed_trlan_info* info,
               cudaStream_t st) {
  auto t_start = std::chrono::steady_clock::now();
  Ctx* ctx = s->ctx;
  const uint64_t n = s->dim;
  const int k = o->k;
  const int kk = (int)std::min<uint64_t>((uint64_t)k, n);
  const int m = (int)std::min<uint64_t>((uint64_t)o->max_basis, n);
  int keep = o->keep > 0 ? o->keep : (m + kk) / 2;
  keep = std::max(kk, std::min(keep, m - 2));
  const int check_every = std::max(1, o->check_every);
  const int max_iter = std::max(1, o->max_iter);
  const size_t eb = sizeof(V);

  // basis V[0..m] (m + 1 vectors), w, rotation target T[0..keep)
  const int n_rot = (m >= 3) ? keep : 0;
  DevBuf vb, cb;
  // slots padded to 32 elements, so that each starts 16-byte aligned
  const uint64_t ld = pad32(n);
  ED_TRY(vb.alloc(ctx, ((size_t)m + 2 + n_rot) * ld * eb));
  ED_TRY(cb.alloc(ctx, coef_bytes(m, 1) + (size_t)kMaxBasis * kMaxBasis * 8 * 4 + (size_t)kMaxBasis * 8 * 8));
  V* Vb = static_cast<V*>(vb.p);
  V* w = Vb + (size_t)(m + 1) * ld;
  V* T = w + ld;  // rotation target, keep vectors of n elements back to back
  Carve cv{static_cast<char*>(cb.p)};
  Coefs c = carve_coefs(cv, m);
  const int ldS = kMaxBasis;
  double* Hp = cv.take<double>((size_t)kMaxBasis * kMaxBasis);
  double* Y = cv.take<double>((size_t)kMaxBasis * kMaxBasis);
  double* Sd = cv.take<double>((size_t)kMaxBasis * ldS);
  float2* Sf = cv.take<float2>((size_t)kMaxBasis * ldS);
  double* theta = cv.take<double>(kMaxBasis);
  double* th = cv.take<double>(kMaxBasis);
  double* sv = cv.take<double>(kMaxBasis);

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
  auto vec = [&](int j) -> V* { return Vb + (size_t)j * ld; };

  k_init_coefs<<<1, 256, 0, st>>>(c, m + 2);
  if (o->v0) {
    ED_TRY_CUDA(cudaMemcpyAsync(w, o->v0, n * eb, cudaMemcpyDeviceToDevice, st));
  } else {
    k_random<V><<<vgrid, 256, 0, st>>>(w, n, o->seed);
  }
  ED_TRY(dot_to(W, (const V*)w, (const V*)w, OP_NORM_INV, 0));
  k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(0), n, c, 0);
  ED_LAUNCH_CHECK();

  // one event pair per basis slot times the H*v launches; read at each check
  std::vector<cudaEvent_t> evs(2 * (size_t)m);
  for (auto& e : evs) ED_TRY_CUDA(cudaEventCreate(&e));
  struct EvGuard {
    std::vector<cudaEvent_t>* v;
    ~EvGuard() {
      for (auto e : *v) cudaEventDestroy(e);
    }
  } evguard{&evs};
  std::vector<int> pending;
  double apply_ms = 0.0;
  auto drain_timers = [&]() {
    for (int q : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, evs[2 * q], evs[2 * q + 1]) == cudaSuccess) apply_ms += ms;
    }
    pending.clear();
  };

  const double thr = 1e-13;
  std::vector<double> h_theta(kMaxBasis), h_last(kMaxBasis), h_res(ED_MAX_K, 0.0);
  int l = 0, size = 0, iters = 0, restarts = 0, injections = 0, n_conv = 0;
  int status = ED_OK;
  bool done = false;
  int j = 0;  // next basis slot to extend from
  while (!done) {
    while (j < m) {
      ED_TRY_CUDA(cudaEventRecord(evs[2 * j], st));
      ED_TRY(apply_h(s, vec(j), w, st));
      ED_TRY_CUDA(cudaEventRecord(evs[2 * j + 1], st));
      pending.push_back(j);
      ED_TRY(dot_to(W, (const V*)vec(j), (const V*)w, OP_ALPHA, j));
      k_lz_update<V><<<vgrid, 256, 0, st>>>(w, vec(j), j > l ? vec(j - 1) : nullptr, n, c, j);
      ED_LAUNCH_CHECK();
      ED_TRY(cgs2(W, (const V*)Vb, ld, j + 1, w));
      ED_TRY(dot_to(W, (const V*)w, (const V*)w, OP_BETA, j + 1, thr));
      k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(j + 1), n, c, j + 1);
      ED_LAUNCH_CHECK();
      ++iters;
      size = ++j;
      if (size < m && ((size - l) % check_every) != 0 && iters < max_iter) continue;
      // first vanished beta: the basis is an invariant subspace up to there
      int ex = -1;
      ED_TRY_CUDA(cudaMemcpyAsync(ctx->h_red, c.exhausted, sizeof(int), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      std::memcpy(&ex, ctx->h_red, sizeof(int));
      drain_timers();
      if (ex >= 0 && ex < size) size = j = ex;  // steps past it are discarded
      // projected eigenproblem of the current basis
      k_tr_project<<<(size * size + 255) / 256, 256, 0, st>>>(Hp, kMaxBasis, size, l, th, sv, c);
      ED_LAUNCH_CHECK();
      ED_TRY(jacobi(st, Hp, size, kMaxBasis, theta, Sd, Sf, ldS, Y));
      const int kc = std::min(kk, size);
      double beta_next = 0.0;
      ED_TRY_CUDA(cudaMemcpyAsync(h_theta.data(), theta, kc * sizeof(double), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaMemcpyAsync(&beta_next, c.beta + size, sizeof(double), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaMemcpy2DAsync(h_last.data(), sizeof(double), Sd + (size - 1), (size_t)ldS * sizeof(double),
                                    sizeof(double), kc, cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      n_conv = 0;
      for (int i = 0; i < kc; ++i) {
        h_res[i] = std::fabs(beta_next * h_last[i]);
        if (h_res[i] <= o->tol * std::max(1.0, std::fabs(h_theta[i])) && n_conv == i) ++n_conv;
      }
      if (ex >= 0) {
        // invariant subspace: its Ritz pairs are exact
        for (int i = 0; i < kc; ++i) h_res[i] = 0.0;
        n_conv = kc;
        if ((uint64_t)size >= n || kc >= kk) {
          done = true;
          break;
        }
        // fewer than k values in it: go on from a fresh direction orthogonal
        // to the basis, uncoupled from it (beta = 0)
        ++injections;
        k_random<V><<<vgrid, 256, 0, st>>>(w, n, o->seed + 7919ull * (uint64_t)injections);
        ED_TRY(cgs2(W, (const V*)Vb, ld, size, w));
        ED_TRY(dot_to(W, (const V*)w, (const V*)w, OP_NORM_INV, 1));
        k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(size), n, c, 1);
        ED_LAUNCH_CHECK();
        const double zero = 0.0;
        const float2 zf = make_float2(0.f, 0.f);
        const int neg = -1;
        ED_TRY_CUDA(cudaMemcpyAsync(c.beta + size, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
        ED_TRY_CUDA(cudaMemcpyAsync(c.nbe_d + size, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
        ED_TRY_CUDA(cudaMemcpyAsync(c.nbe_f + size, &zf, sizeof(float2), cudaMemcpyHostToDevice, st));
        ED_TRY_CUDA(cudaMemcpyAsync(c.exhausted, &neg, sizeof(int), cudaMemcpyHostToDevice, st));
        ED_TRY_CUDA(cudaStreamSynchronize(st));
        continue;  // j == size: the next step starts from the new vector (a full basis restarts first)
      }
      if (kc >= kk && n_conv >= kk) {
        done = true;
        break;
      }
      if (iters >= max_iter) {
        status = ED_ERR_NOT_CONVERGED;
        done = true;
        break;
      }
    }
    if (done) break;
    // basis full: keep the `keep` lowest Ritz vectors and the residual direction
    if (n_rot == 0) {
      status = ED_ERR_NOT_CONVERGED;
      break;
    }
    for (int i0 = 0; i0 < keep; i0 += 8)
      k_ritz<V, 8><<<vgrid, 256, 0, st>>>(Vb, ld, m, Sd, Sf, ldS, i0, std::min(8, keep - i0), T, n, 0);
    ED_LAUNCH_CHECK();
    ED_TRY_CUDA(cudaMemcpy2DAsync(Vb, ld * eb, T, n * eb, n * eb, keep, cudaMemcpyDeviceToDevice, st));
    ED_TRY_CUDA(cudaMemcpyAsync(vec(keep), vec(m), n * eb, cudaMemcpyDeviceToDevice, st));
    k_tr_keep<<<1, 128, 0, st>>>(theta, Sd, ldS, m, keep, c, th, sv);
    ED_LAUNCH_CHECK();
    l = j = keep;
    ++restarts;
  }
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  drain_timers();

  const int kc = std::min(kk, size);
  for (int i = 0; i < kc; ++i) evals[i] = h_theta[i];
  for (int i = kc; i < k; ++i) evals[i] = NAN;
  if (evecs && kc > 0) {
    // Sd holds the eigenvectors of the last projected matrix (size `size`)
    V* out = static_cast<V*>(evecs);
    for (int i0 = 0; i0 < kc; i0 += 8)
      k_ritz<V, 8><<<vgrid, 256, 0, st>>>(Vb, ld, size, Sd, Sf, ldS, i0, std::min(8, kc - i0), out, n, 0);
    ED_LAUNCH_CHECK();
  }
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->iters = iters;
    info->restarts = restarts;
    info->n_converged = std::min(n_conv, kc);
    for (int i = 0; i < ED_MAX_K; ++i) info->residual[i] = (i < kc) ? h_res[i] : 0.0;
    info->apply_ms = apply_ms;
    info->basis_bytes = ((size_t)m + 2 + n_rot) * ld * eb;
    info->total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  }
  if (status != ED_OK) set_error("thick-restart Lanczos did not converge in %d products", max_iter);
  return status;
}

}  // namespace

int trlan_run(Sector* s, const ed_trlan_opts* o, double* evals, void* evecs, ed_trlan_info* info,
              cudaStream_t st) {
  if (!o || !evals) ED_INVALID("NULL argument");
  if (o->k < 1 || o->k > ED_MAX_K) ED_INVALID("k must be in 1..%d", ED_MAX_K);
  if (!(o->tol > 0.0)) ED_INVALID("tol must be positive");
  if (o->max_basis > ED_MAX_BASIS) ED_INVALID("max_basis must be at most %d", ED_MAX_BASIS);
  const uint64_t n = s->dim;
  const uint64_t kk = std::min<uint64_t>((uint64_t)o->k, n);
  if ((uint64_t)o->max_basis < std::min<uint64_t>(kk + 2, n))
    ED_INVALID("max_basis (%d) must be at least k + 2 (or the sector dimension)", o->max_basis);
  if (o->keep != 0 && (o->keep < (int)kk || o->keep > o->max_basis - 2))
    ED_INVALID("keep must be 0 or in k..max_basis-2");
  switch (s->prec) {
    case ED_PREC_FP64: return trlan_impl<double>(s, o, evals, evecs, info, st);
    case ED_PREC_DF64: return trlan_impl<float2>(s, o, evals, evecs, info, st);
    case ED_PREC_FP32: return trlan_impl<float>(s, o, evals, evecs, info, st);
  }
  ED_INVALID("unknown precision");
}

}  // namespace ed
