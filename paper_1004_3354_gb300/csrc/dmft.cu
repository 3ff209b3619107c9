// One DMFT self-consistency update for the one-band Hubbard model (Sec. 2: the
// lattice problem is reduced to the Anderson impurity of Eq. 2, whose
// Green's function closes the loop; Sec. 3.2 runs it on the square lattice).
// From the impurity G(i w_n) of the AIM with level eps_d and bath (eps_k, V_k):
//
//   Delta(z)   = sum_k V_k^2 / (z - eps_k)              bath hybridisation
//   Sigma      = z - eps_d - Delta - 1 / G_imp          impurity self-energy
//   G_loc      = sum_j w_j / (z + mu - e_j - Sigma)     lattice local Green's function
//   Delta_new  = z - eps_d - Sigma - 1 / G_loc          new Weiss field, as a hybridisation
//
// at z = i w_n on the device (one block per frequency, its threads over the
// caller's band-energy quadrature e_j, w_j), then the new bath as the
// least-squares fit of Delta_new on the first n_fit frequencies by
// Levenberg-Marquardt on the host (2 n_bath parameters).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr int kDT = 256;

// 1 / (c + i d) by Smith's (1962) scaled division.
__device__ __forceinline__ double2 crecip_s(double c, double d) {
  if (fabs(c) >= fabs(d)) {
    double r = d / c, den = c + d * r;
    return make_double2(1.0 / den, -r / den);
  }
  double r = c / d, den = c * r + d;
  return make_double2(r / den, -1.0 / den);
}

__global__ void __launch_bounds__(kDT) k_dmft_update(int n_w, double beta, const double2* __restrict__ G_imp,
                                                    double eps_d, double mu, int n_bath,
                                                    const double* __restrict__ eps, const double* __restrict__ V,
                                                    int n_e, const double* __restrict__ e,
                                                    const double* __restrict__ wt, double2* __restrict__ sigma,
                                                    double2* __restrict__ gloc, double2* __restrict__ dnew) {
  __shared__ double2 sig_s;
  __shared__ double rre[kDT / 32], rim[kDT / 32];
  const int n = blockIdx.x;
  if (n >= n_w) return;
  const double wn = (2.0 * n + 1.0) * 3.14159265358979323846 / beta;
  if (threadIdx.x == 0) {
    double dre = 0.0, dim = 0.0;  // Delta(i w_n)
    for (int k = 0; k < n_bath; ++k) {
      const double2 r = crecip_s(-eps[k], wn);
      dre += V[k] * V[k] * r.x;
      dim += V[k] * V[k] * r.y;
    }
    const double2 g = G_imp[n];
    const double den = g.x * g.x + g.y * g.y;
    const double2 ig = make_double2(g.x / den, -g.y / den);  // 1 / G_imp
    sig_s = make_double2(-eps_d - dre - ig.x, wn - dim - ig.y);
  }
  __syncthreads();
  const double2 sg = sig_s;
  double are = 0.0, aim = 0.0;
  for (int j = threadIdx.x; j < n_e; j += kDT) {
    const double2 r = crecip_s(mu - e[j] - sg.x, wn - sg.y);
    are += wt[j] * r.x;
    aim += wt[j] * r.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    are += __shfl_xor_sync(0xffffffffu, are, o);
    aim += __shfl_xor_sync(0xffffffffu, aim, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rre[threadIdx.x >> 5] = are;
    rim[threadIdx.x >> 5] = aim;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gre = 0.0, gim = 0.0;
    for (int q = 0; q < kDT / 32; ++q) {
      gre += rre[q];
      gim += rim[q];
    }
    const double den = gre * gre + gim * gim;
    sigma[n] = sg;
    gloc[n] = make_double2(gre, gim);
    dnew[n] = make_double2(-eps_d - sg.x - gre / den, wn - sg.y + gim / den);
  }
}

using cplx = std::complex<double>;

double bath_chi2(const std::vector<cplx>& z, const std::vector<cplx>& target, const std::vector<double>& p, int nb) {
  double s = 0.0;
  for (size_t n = 0; n < z.size(); ++n) {
    cplx d = 0.0;
    for (int k = 0; k < nb; ++k) d += p[nb + k] * p[nb + k] / (z[n] - p[k]);
    s += std::norm(target[n] - d);
  }
  return s / (double)z.size();
}

// Solve (A) x = b for symmetric positive definite A (size m) by Cholesky;
// false if A is not positive definite.
bool chol_solve(std::vector<double> A, std::vector<double> b, int m, std::vector<double>& x) {
  for (int j = 0; j < m; ++j) {
    double d = A[j * m + j];
    for (int k = 0; k < j; ++k) d -= A[j * m + k] * A[j * m + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double v = A[i * m + j];
      for (int k = 0; k < j; ++k) v -= A[i * m + k] * A[j * m + k];
      A[i * m + j] = v / d;
    }
  }
  for (int i = 0; i < m; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= A[i * m + k] * b[k];
    b[i] = v / A[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < m; ++k) v -= A[k * m + i] * b[k];
    b[i] = v / A[i * m + i];
  }
  x = b;
  return true;
}

// Levenberg-Marquardt fit of sum_k V_k^2 / (z - eps_k) to target on z; p = (eps, V).
double fit_bath_lm(const std::vector<cplx>& z, const std::vector<cplx>& target, std::vector<double>& p, int nb) {
  const int np = 2 * nb, nz = (int)z.size();
  double chi = bath_chi2(z, target, p, nb);
  double lam = 1e-3;
  std::vector<double> A(np * np), g(np), J(np), step;
  for (int it = 0; it < 2000; ++it) {
    std::fill(A.begin(), A.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    for (int n = 0; n < nz; ++n) {
      cplx d = 0.0;
      std::vector<cplx> dj(np);
      for (int k = 0; k < nb; ++k) {
        const cplx r = 1.0 / (z[n] - p[k]);
        const double v = p[nb + k];
        d += v * v * r;
        dj[k] = v * v * r * r;   // d Delta / d eps_k
        dj[nb + k] = 2.0 * v * r;  // d Delta / d V_k
      }
      const cplx res = d - target[n];  // residual of the fit
      for (int a = 0; a < np; ++a) {
        g[a] += (std::conj(dj[a]) * res).real();
        for (int b = 0; b <= a; ++b) A[a * np + b] += (std::conj(dj[a]) * dj[b]).real();
      }
    }
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < a; ++b) A[b * np + a] = A[a * np + b];
    bool moved = false;
    while (lam < 1e16) {
      std::vector<double> M = A, rhs(np);
      for (int a = 0; a < np; ++a) {
        M[a * np + a] += lam * std::max(A[a * np + a], 1e-300);
        rhs[a] = -g[a];
      }
      if (chol_solve(M, rhs, np, step)) {
        std::vector<double> q = p;
        for (int a = 0; a < np; ++a) q[a] += step[a];
        const double c2 = bath_chi2(z, target, q, nb);
        if (c2 < chi) {
          const double rel = (chi - c2) / std::max(chi, 1e-300);
          p = q;
          chi = c2;
          lam = std::max(lam / 3.0, 1e-15);
          moved = true;
          if (rel < 1e-13) return chi;
          break;
        }
      }
      lam *= 4.0;
    }
    if (!moved) break;
  }
  return chi;
}

}  // namespace

int dmft_update(Ctx* ctx, int n_w, double beta, const double* G_imp, double eps_d, double mu, int n_bath,
                const double* eps_in, const double* V_in, int n_e, const double* e, const double* w, int n_fit,
                double* eps_out, double* V_out, double* chi2, double* sigma, double* G_loc, double* delta_new,
                cudaStream_t st) {
  if (!G_imp || !eps_in || !V_in || !e || !w || !eps_out || !V_out) ED_INVALID("NULL argument");
  if (n_w < 1 || !(beta > 0.0)) ED_INVALID("n_w must be >= 1 and beta > 0");
  if (n_bath < 1 || n_bath > ED_MAX_SITES) ED_INVALID("n_bath must be in 1..%d", ED_MAX_SITES);
  if (n_e < 1) ED_INVALID("n_e must be >= 1");
  if (n_fit < 1 || n_fit > n_w) ED_INVALID("n_fit must be in 1..n_w");
  for (int n = 0; n < n_w; ++n)
    if (!(std::isfinite(G_imp[2 * n]) && std::isfinite(G_imp[2 * n + 1])) ||
        G_imp[2 * n] * G_imp[2 * n] + G_imp[2 * n + 1] * G_imp[2 * n + 1] == 0.0)
      ED_INVALID("G_imp[%d] is zero or not finite", n);
  // device work: inputs, then the three outputs
  const size_t nb = (size_t)n_bath, ne = (size_t)n_e, nw = (size_t)n_w;
  const size_t bytes = sizeof(double) * (2 * nw + 2 * nb + 2 * ne + 6 * nw);
  void* buf = nullptr;
  ED_TRY(dev_alloc(ctx, &buf, bytes));
  struct Free {
    Ctx* c;
    void* p;
    size_t b;
    ~Free() { dev_free(c, p, b); }
  } fb{ctx, buf, bytes};
  double* dG = static_cast<double*>(buf);
  double* dEps = dG + 2 * nw;
  double* dV = dEps + nb;
  double* dE = dV + nb;
  double* dW = dE + ne;
  double* dOut = dW + ne;  // sigma, gloc, dnew (complex each)
  ED_TRY_CUDA(cudaMemcpyAsync(dG, G_imp, sizeof(double) * 2 * nw, cudaMemcpyHostToDevice, st));
  ED_TRY_CUDA(cudaMemcpyAsync(dEps, eps_in, sizeof(double) * nb, cudaMemcpyHostToDevice, st));
  ED_TRY_CUDA(cudaMemcpyAsync(dV, V_in, sizeof(double) * nb, cudaMemcpyHostToDevice, st));
  ED_TRY_CUDA(cudaMemcpyAsync(dE, e, sizeof(double) * ne, cudaMemcpyHostToDevice, st));
  ED_TRY_CUDA(cudaMemcpyAsync(dW, w, sizeof(double) * ne, cudaMemcpyHostToDevice, st));
  double2* o = reinterpret_cast<double2*>(dOut);
  k_dmft_update<<<n_w, kDT, 0, st>>>(n_w, beta, reinterpret_cast<const double2*>(dG), eps_d, mu, n_bath, dEps, dV,
                                     n_e, dE, dW, o, o + nw, o + 2 * nw);
  ED_LAUNCH_CHECK();
  std::vector<double> h(6 * nw);
  ED_TRY_CUDA(cudaMemcpyAsync(h.data(), dOut, sizeof(double) * 6 * nw, cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  if (sigma) std::copy(h.begin(), h.begin() + 2 * nw, sigma);
  if (G_loc) std::copy(h.begin() + 2 * nw, h.begin() + 4 * nw, G_loc);
  if (delta_new) std::copy(h.begin() + 4 * nw, h.end(), delta_new);
  // bath fit on the first n_fit Matsubara points
  std::vector<cplx> z(n_fit), target(n_fit);
  for (int n = 0; n < n_fit; ++n) {
    z[n] = cplx(0.0, (2.0 * n + 1.0) * M_PI / beta);
    target[n] = cplx(h[4 * nw + 2 * n], h[4 * nw + 2 * n + 1]);
  }
  std::vector<double> p(2 * nb);
  for (size_t k = 0; k < nb; ++k) {
    p[k] = eps_in[k];
    p[nb + k] = V_in[k];
  }
  const double c2 = fit_bath_lm(z, target, p, n_bath);
  for (size_t k = 0; k < nb; ++k) {
    eps_out[k] = p[k];
    V_out[k] = std::fabs(p[nb + k]);
  }
  if (chi2) *chi2 = c2;
  return ED_OK;
}

}  // namespace ed
