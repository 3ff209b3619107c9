// Green's function from the lowest states by Lanczos continued fractions
// (Eq. 3; the sum over final states mu is carried by the Lanczos
// tridiagonalisation started from c+|nu> and c|nu>).  Sec. 2 notes that at
// large beta only the lowest states carry weight; Sec. 4 keeps the states
// whose Boltzmann factor exceeds a cutoff.
//
//   G(z) = sum_nu w_nu [ n+ / (z + E_nu - a_0 - b_1^2 / (z + E_nu - a_1 - ...))
//                      + n- / (z - E_nu + a_0 - b_1^2 / (z - E_nu + a_1 - ...)) ]
//   w_nu = e^{-beta (E_nu - E_min)} / Z,
//
// at the Matsubara points z = i w_n, w_n = (2n+1) pi / beta, or at any given
// complex z off the real axis: z = w + i eta gives the real-frequency spectral
// function A(w) = -Im G(w + i eta) / pi that Figs. 3 and 5 plot.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

// 1 / (c + i d) by Smith's (1962) scaled division.
__device__ __forceinline__ double2 crecip(double c, double d) {
  if (fabs(c) >= fabs(d)) {
    double r = d / c, den = c + d * r;
    return make_double2(1.0 / den, -r / den);
  }
  double r = c / d, den = c * r + d;
  return make_double2(r / den, -1.0 / den);
}

// One (state, part) contribution per launch; thread = frequency index.
// sgn = +1 particle part (z + E - H), -1 hole part (z - E + H).  z == NULL:
// Matsubara points i w_n; otherwise z[n] = (re, im).
__global__ void k_cf_accum(double2* __restrict__ G, int n_w, double beta, const double* __restrict__ a,
                           const double* __restrict__ b, int L, double n2, const double* __restrict__ E,
                           int n_states, int nu, int sgn, const double2* __restrict__ z) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_w || L <= 0) return;
  double Emin = E[0];
  for (int i = 1; i < n_states; ++i) Emin = fmin(Emin, E[i]);
  double Z = 0.0;
  for (int i = 0; i < n_states; ++i) Z += exp(-beta * (E[i] - Emin));
  double w = exp(-beta * (E[nu] - Emin)) / Z;
  const double zr = z ? z[n].x : 0.0;
  const double zi = z ? z[n].y : (2.0 * n + 1.0) * 3.14159265358979323846 / beta;
  // particle: re(z') = Re z + E - a_i ; hole: re(z') = Re z - E + a_i ; im(z') = Im z
  double En = E[nu];
  double2 g = crecip(zr + (sgn > 0 ? (En - a[L - 1]) : (-En + a[L - 1])), zi);
  for (int i = L - 2; i >= 0; --i) {
    double re = zr + (sgn > 0 ? (En - a[i]) : (-En + a[i])) - b[i + 1] * b[i + 1] * g.x;
    double im = zi - b[i + 1] * b[i + 1] * g.y;
    g = crecip(re, im);
  }
  G[n].x += w * n2 * g.x;
  G[n].y += w * n2 * g.y;
}

struct SectorCache {
  Ctx* ctx;
  const ed_model* m;
  int prec;
  std::map<std::pair<int, int>, std::unique_ptr<Sector>> cache;
  int get(int nu, int nd, Sector** out) {
    auto key = std::make_pair(nu, nd);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second.get();
      return ED_OK;
    }
    std::unique_ptr<Sector> s(new Sector());
    int st = build_sector(ctx, m, nu, nd, prec, s.get());
    if (st == ED_OK) st = build_fast(s.get());  // the fast row kernel where the sector allows it
    if (st != ED_OK) {
      free_sector(s.get());
      return st;
    }
    *out = s.get();
    cache[key] = std::move(s);
    return ED_OK;
  }
  ~SectorCache() {
    for (auto& kv : cache) free_sector(kv.second.get());
  }
};

}  // namespace

// Add one (state, part) continued fraction to G on `st` (used by the server).
int greens_accumulate(double2* dG, int n_w, double beta, const double* da, const double* db, int L, double n2,
                      const double* dE, int n_states, int nu, int sgn, cudaStream_t st) {
  k_cf_accum<<<(n_w + 127) / 128, 128, 0, st>>>(dG, n_w, beta, da, db, L, n2, dE, n_states, nu, sgn, nullptr);
  ED_LAUNCH_CHECK();
  return ED_OK;
}

int greens_cf_run(Ctx* ctx, const ed_model* m, int prec, int n_states, const ed_state* states, double beta,
                  int n_w, const double* z, int orbital, int spin, int depth, double boltz_cut, double* G,
                  double* coeffs, cudaStream_t st) {
  ED_TRY(validate_model(m));
  if (n_states < 1 || !states) ED_INVALID("no states");
  if (!(beta > 0.0)) ED_INVALID("beta must be positive");
  if (n_w < 1 || !G) ED_INVALID("n_w must be positive and G non-NULL");
  if (z)
    for (int n = 0; n < n_w; ++n)
      if (!std::isfinite(z[2 * n]) || !(z[2 * n + 1] > 0.0))
        ED_INVALID("z[%d] = (%g, %g): frequencies need Im z > 0", n, z[2 * n], z[2 * n + 1]);
  if (depth < 1) ED_INVALID("depth must be >= 1");
  if (spin != ED_SPIN_UP && spin != ED_SPIN_DN) ED_INVALID("spin must be 0 or 1");
  if (orbital < 0 || orbital >= m->n_s) ED_INVALID("orbital outside 0..n_s-1");
  double Emin = states[0].E;
  for (int i = 0; i < n_states; ++i) {
    if (!states[i].vec) ED_INVALID("state %d has no vector", i);
    Emin = std::min(Emin, states[i].E);
  }
  SectorCache sc{ctx, m, prec, {}};
  double2* dG = nullptr;
  double* dE = nullptr;
  double* dab = nullptr;
  ED_TRY(dev_alloc_n(ctx, &dG, (size_t)n_w));
  struct Free {
    Ctx* c;
    void* p;
    size_t b;
    ~Free() {
      if (p) dev_free(c, p, b);
    }
  } f1{ctx, dG, sizeof(double2) * n_w};
  ED_TRY(dev_alloc_n(ctx, &dE, (size_t)n_states));
  Free f2{ctx, dE, sizeof(double) * n_states};
  ED_TRY(dev_alloc_n(ctx, &dab, (size_t)2 * depth));
  Free f3{ctx, dab, sizeof(double) * 2 * depth};
  double2* dz = nullptr;
  if (z) {
    ED_TRY(dev_alloc_n(ctx, &dz, (size_t)n_w));
    ED_TRY_CUDA(cudaMemcpyAsync(dz, z, sizeof(double2) * n_w, cudaMemcpyHostToDevice, st));
  }
  Free f4{ctx, dz, z ? sizeof(double2) * n_w : 0};
  ED_TRY_CUDA(cudaMemsetAsync(dG, 0, sizeof(double2) * n_w, st));
  std::vector<double> hE(n_states);
  for (int i = 0; i < n_states; ++i) hE[i] = states[i].E;
  ED_TRY_CUDA(cudaMemcpyAsync(dE, hE.data(), sizeof(double) * n_states, cudaMemcpyHostToDevice, st));
  std::vector<double> ha(depth), hb(depth);
  size_t rec = 2 + 2 * (size_t)depth;
  int kept = 0;
  for (int nu = 0; nu < n_states; ++nu) {
    if (std::exp(-beta * (states[nu].E - Emin)) < boltz_cut) continue;
    const ed_state& S = states[nu];
    Sector* src = nullptr;
    ED_TRY(sc.get(S.n_up, S.n_dn, &src));
    for (int part = 0; part < 2; ++part) {
      bool dag = (part == 0);
      int tu = S.n_up + ((spin == ED_SPIN_UP) ? (dag ? 1 : -1) : 0);
      int td = S.n_dn + ((spin == ED_SPIN_DN) ? (dag ? 1 : -1) : 0);
      double n2 = 0.0;
      int L = 0;
      std::fill(ha.begin(), ha.end(), 0.0);
      std::fill(hb.begin(), hb.end(), 0.0);
      if (tu >= 0 && tu <= m->n_s && td >= 0 && td <= m->n_s) {
        Sector* dst = nullptr;
        ED_TRY(sc.get(tu, td, &dst));
        void* phi = nullptr;
        size_t pb = dst->dim * elem_bytes(prec);
        ED_TRY(dev_alloc(ctx, &phi, pb));
        Free fp{ctx, phi, pb};
        ED_TRY(apply_cop(src, dst, orbital, spin, dag, S.vec, phi, st));
        ED_TRY(lanczos_coeffs(dst, phi, depth, &n2, ha.data(), hb.data(), &L, st));
        if (L > 0 && n2 > 0.0) {
          ED_TRY_CUDA(cudaMemcpyAsync(dab, ha.data(), sizeof(double) * depth, cudaMemcpyHostToDevice, st));
          ED_TRY_CUDA(cudaMemcpyAsync(dab + depth, hb.data(), sizeof(double) * depth, cudaMemcpyHostToDevice, st));
          k_cf_accum<<<(n_w + 127) / 128, 128, 0, st>>>(dG, n_w, beta, dab, dab + depth, L, n2, dE, n_states, nu,
                                                       dag ? 1 : -1, dz);
          ED_LAUNCH_CHECK();
          ED_TRY_CUDA(cudaStreamSynchronize(st));  // ha/hb are reused
        }
      }
      if (coeffs) {
        double* r = coeffs + ((size_t)kept * 2 + part) * rec;
        r[0] = n2;
        r[1] = (double)L;
        for (int i = 0; i < depth; ++i) {
          r[2 + i] = ha[i];
          r[2 + depth + i] = hb[i];
        }
      }
    }
    ++kept;
  }
  ED_TRY_CUDA(cudaMemcpyAsync(G, dG, sizeof(double2) * n_w, cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  return ED_OK;
}

}  // namespace ed
