// Tridiagonal eigensolver used by the Lanczos drivers (internal header):
// Sturm-sequence multisection for the k lowest eigenvalues (one warp per
// value), inverse iteration with tridiagonal Gaussian elimination and partial
// pivoting for the eigenvectors, then Gram-Schmidt among (nearly) equal
// eigenvalues.  All in FP64.
#pragma once

#include "ed_internal.h"

namespace ed {

// Block-wide sum, result valid in thread 0.
__device__ inline double tri_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    v = (lane < nw) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// Sturm count: number of eigenvalues of T (alpha[0..m), beta[1..m)) below x.
__device__ inline int sturm(const double* __restrict__ a, const double* __restrict__ b, int m, double x,
                     double pivmin) {
  int cnt = 0;
  double q = a[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = (a[i] - x) - b[i] * b[i] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Eigenvalue `blockIdx.x` (ascending) by 32-way multisection, one warp per value.
__device__ inline void tri_eig_one(const double* __restrict__ a, const double* __restrict__ b, int m, int i,
                                   double* __restrict__ theta) {
  int lane = threadIdx.x;
  double lo = a[0], hi = a[0], bmax = 0.0;
  for (int r = 0; r < m; ++r) {
    double off = (r > 0 ? fabs(b[r]) : 0.0) + (r + 1 < m ? fabs(b[r + 1]) : 0.0);
    lo = fmin(lo, a[r] - off);
    hi = fmax(hi, a[r] + off);
    if (r > 0) bmax = fmax(bmax, fabs(b[r]));
  }
  double scale = fmax(fabs(lo), fabs(hi));
  double pivmin = fmax(1e-300, 1e-290 * bmax * bmax);
  lo -= 1e-14 * scale + 1e-300;
  hi += 1e-14 * scale + 1e-300;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
    double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    int c = sturm(a, b, m, x, pivmin);
    // first lane whose point has more than i eigenvalues below it
    unsigned above = __ballot_sync(0xffffffffu, c > i);
    int f = above ? __ffs(above) - 1 : 32;
    double nlo = (f == 0) ? lo : lo + (hi - lo) * (double)f / 33.0;
    double nhi = (f == 32) ? hi : lo + (hi - lo) * (double)(f + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) theta[i] = 0.5 * (lo + hi);
}

// Inverse iteration for eigenvector blockIdx.x: solve (T - theta I) x = x_prev
// by tridiagonal Gaussian elimination with partial pivoting (row interchanges
// as in LAPACK's gttrf/gtts2), three sweeps.  work holds 6*ldS doubles per
// eigenvector.  Output S[i*ldS + j], j < m, normalised, largest entry positive.
__device__ inline void tri_vec_one(const double* __restrict__ a, const double* __restrict__ b, int m,
                                   const double* __restrict__ theta, double* __restrict__ S, int ldS,
                                   double* __restrict__ work, int k) {
  double* x = work + (size_t)k * 6 * ldS;
  double* dl = x + ldS;
  double* d = dl + ldS;
  double* du = d + ldS;
  double* du2 = du + ldS;
  double* piv = du2 + ldS;
  double* s = S + (size_t)k * ldS;
  const double th = theta[k];
  double anorm = 0.0;
  for (int r = 0; r < m; ++r)
    anorm = fmax(anorm, fabs(a[r]) + (r > 0 ? fabs(b[r]) : 0.0) + (r + 1 < m ? fabs(b[r + 1]) : 0.0));
  const double tiny = 2.2e-16 * fmax(anorm, 1e-300);
  for (int r = 0; r < m; ++r) {
    d[r] = a[r] - th;
    du[r] = (r + 1 < m) ? b[r + 1] : 0.0;
    dl[r] = (r + 1 < m) ? b[r + 1] : 0.0;  // subdiagonal (symmetric)
    du2[r] = 0.0;
    piv[r] = 0.0;
  }
  for (int r = 0; r + 1 < m; ++r) {
    if (fabs(d[r]) >= fabs(dl[r])) {
      double f = (d[r] != 0.0) ? dl[r] / d[r] : 0.0;
      dl[r] = f;
      d[r + 1] -= f * du[r];
    } else {
      double f = d[r] / dl[r];
      d[r] = dl[r];
      dl[r] = f;
      double t = du[r];
      du[r] = d[r + 1];
      d[r + 1] = t - f * d[r + 1];
      if (r + 2 < m) {
        du2[r] = du[r + 1];
        du[r + 1] = -f * du[r + 1];
      }
      piv[r] = 1.0;
    }
  }
  for (int r = 0; r < m; ++r)
    if (fabs(d[r]) < tiny) d[r] = (d[r] < 0 ? -tiny : tiny);
  for (int r = 0; r < m; ++r) x[r] = 1.0 + 0.01 * (double)((r * 7919 + k * 104729) % 97) / 97.0;
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int r = 0; r + 1 < m; ++r) {
      if (piv[r] == 0.0) {
        x[r + 1] -= dl[r] * x[r];
      } else {
        double t = x[r];
        x[r] = x[r + 1];
        x[r + 1] = t - dl[r] * x[r];
      }
    }
    x[m - 1] /= d[m - 1];
    if (m > 1) x[m - 2] = (x[m - 2] - du[m - 2] * x[m - 1]) / d[m - 2];
    for (int r = m - 3; r >= 0; --r) x[r] = (x[r] - du[r] * x[r + 1] - du2[r] * x[r + 2]) / d[r];
    double mx = 0.0;
    for (int r = 0; r < m; ++r) mx = fmax(mx, fabs(x[r]));
    double inv = mx > 0 ? 1.0 / mx : 0.0;
    double nrm = 0.0;
    for (int r = 0; r < m; ++r) {
      x[r] *= inv;
      nrm += x[r] * x[r];
    }
    inv = nrm > 0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int r = 0; r < m; ++r) x[r] *= inv;
  }
  int big = 0;
  for (int r = 1; r < m; ++r)
    if (fabs(x[r]) > fabs(x[big])) big = r;
  double sg = x[big] < 0 ? -1.0 : 1.0;
  for (int r = 0; r < m; ++r) s[r] = sg * x[r];
}

// Orthogonalise eigenvectors of (nearly) equal eigenvalues in order, then
// residual estimates |beta_m s_{m-1,i}| and double-float copies.
__device__ inline void tri_finish_block(const double* __restrict__ theta, int k, int m, double beta_m,
                                        double* __restrict__ S, int ldS, float2* __restrict__ Sf,
                                        double* __restrict__ resid) {
  __shared__ double sh[32];
  double scale = 0.0;
  for (int i = 0; i < k; ++i) scale = fmax(scale, fabs(theta[i]));
  for (int i = 0; i < k; ++i) {
    double* si = S + (uint64_t)i * ldS;
    for (int j = 0; j < i; ++j) {
      if (fabs(theta[i] - theta[j]) > 1e-9 * fmax(scale, 1.0)) continue;
      double* sj = S + (uint64_t)j * ldS;
      double p = 0.0;
      for (int r = threadIdx.x; r < m; r += blockDim.x) p += si[r] * sj[r];
      p = tri_block_sum(p, sh);
      if (threadIdx.x == 0) sh[0] = p;
      __syncthreads();
      p = sh[0];
      __syncthreads();
      for (int r = threadIdx.x; r < m; r += blockDim.x) si[r] -= p * sj[r];
      __syncthreads();
      double q = 0.0;
      for (int r = threadIdx.x; r < m; r += blockDim.x) q += si[r] * si[r];
      q = tri_block_sum(q, sh);
      if (threadIdx.x == 0) sh[0] = q;
      __syncthreads();
      q = sh[0];
      __syncthreads();
      double inv = q > 0 ? 1.0 / sqrt(q) : 0.0;
      for (int r = threadIdx.x; r < m; r += blockDim.x) si[r] *= inv;
      __syncthreads();
    }
  }
  for (int i = 0; i < k; ++i) {
    for (int r = threadIdx.x; r < m; r += blockDim.x) Sf[(uint64_t)i * ldS + r] = df_from_double(S[(uint64_t)i * ldS + r]);
    if (threadIdx.x == 0) resid[i] = fabs(beta_m * S[(uint64_t)i * ldS + m - 1]);
  }
}

}  // namespace ed
