// Sector set-up on the device: spin-string bases (combinatorial ranking and
// unranking), one-body hop tables with fermion signs, diagonal tables,
// spin-flip / pair-hop maps, and the c+ / c maps between neighbour sectors.
//
// This replaces building the stored Hamiltonian (the T_setup column of
// Table 1): the work is O(D_up + D_dn) instead of O(nnz).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr int kB = 33;  // stride of the binomial table C[n * kB + k]

__device__ __forceinline__ uint32_t rank_of(uint32_t s, const uint32_t* __restrict__ C) {
  uint32_t r = 0;
  int k = 1;
  while (s) {
    int p = __ffs(s) - 1;
    r += C[p * kB + k];
    ++k;
    s &= s - 1;
  }
  return r;
}

__device__ __forceinline__ uint32_t unrank(uint32_t r, int n_s, int n,
                                           const uint32_t* __restrict__ C) {
  uint32_t s = 0;
  for (int k = n; k >= 1; --k) {
    int p = k - 1;
    while (p + 1 < n_s && C[(p + 1) * kB + k] <= r) ++p;
    s |= 1u << p;
    r -= C[p * kB + k];
  }
  return s;
}

// Bits strictly between sites i and j.
__device__ __forceinline__ uint32_t between(int i, int j) {
  int lo = min(i, j), hi = max(i, j);
  uint32_t below_hi = (hi >= 32) ? 0xffffffffu : ((1u << hi) - 1u);
  uint32_t upto_lo = (lo + 1 >= 32) ? 0xffffffffu : ((1u << (lo + 1)) - 1u);
  return below_hi & ~upto_lo;
}

struct ModelArgs {
  int n_s, M, orb0;
  double UpmJ;            // U' - J (same-spin inter-orbital)
  const double* T;        // device n_s * n_s
};

// Basis string, one-spin diagonal part and hop count of every rank.
__global__ void k_spin_count(ModelArgs m, int n, uint32_t D, const uint32_t* __restrict__ C,
                             uint32_t* __restrict__ basis, double* __restrict__ e,
                             uint32_t* __restrict__ count) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D) return;
  uint32_t s = unrank(r, m.n_s, n, C);
  basis[r] = s;
  double acc = 0.0;
  for (int i = 0; i < m.n_s; ++i)
    if ((s >> i) & 1u) acc += m.T[i * m.n_s + i];
  for (int a = m.orb0; a < m.orb0 + m.M; ++a)
    for (int b = a + 1; b < m.orb0 + m.M; ++b)
      if (((s >> a) & 1u) && ((s >> b) & 1u)) acc += m.UpmJ;
  e[r] = acc;
  uint32_t c = 0;
  for (int i = 0; i < m.n_s; ++i) {
    if (!((s >> i) & 1u)) continue;
    for (int j = 0; j < m.n_s; ++j)
      if (j != i && !((s >> j) & 1u) && m.T[i * m.n_s + j] != 0.0) ++c;
  }
  count[r] = c;
}

constexpr int kMaxLocal = 256;

// Hop entries of every rank: moving the electron at i to the empty site j gives
// <s|T_ij c+_i c_j|s - i + j> = T_ij (-1)^{popcount(s & between(i, j))}; sorted
// by target rank.
__global__ void k_spin_fill(ModelArgs m, uint32_t D, const uint32_t* __restrict__ C,
                            const uint32_t* __restrict__ basis, const uint32_t* __restrict__ ptr,
                            uint32_t* __restrict__ tgt, double* __restrict__ val) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D) return;
  uint32_t s = basis[r];
  uint32_t t[kMaxLocal];
  double v[kMaxLocal];
  int c = 0;
  for (int i = 0; i < m.n_s; ++i) {
    if (!((s >> i) & 1u)) continue;
    for (int j = 0; j < m.n_s; ++j) {
      if (j == i || ((s >> j) & 1u)) continue;
      double tij = m.T[i * m.n_s + j];
      if (tij == 0.0) continue;
      uint32_t s2 = s ^ (1u << i) ^ (1u << j);
      double sg = (__popc(s & between(i, j)) & 1) ? -1.0 : 1.0;
      uint32_t rt = rank_of(s2, C);
      // insertion by target rank
      int k = c++;
      while (k > 0 && t[k - 1] > rt) {
        t[k] = t[k - 1];
        v[k] = v[k - 1];
        --k;
      }
      t[k] = rt;
      v[k] = tij * sg;
    }
  }
  uint32_t o = ptr[r];
  for (int k = 0; k < c; ++k) {
    tgt[o + k] = t[k];
    val[o + k] = v[k];
  }
}

// Cross diagonal tables: W_c[a][b] = sum_{i in chunk c} U_i a_i b_i
//                                    + [c == oc] U' sum_{m != m'} a_m b_m'.
// Chunk c covers sites w_lo + 8c ...; the M orbitals occupy bits o0 .. o0 + M - 1
// of chunk oc.
__global__ void k_cross(int n_chunks, int4 bits, uint4 off, const double* __restrict__ U, int w_lo,
                        int M, int oc, int o0, double Up, uint32_t total, double* __restrict__ W) {
  uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int bw[4] = {bits.x, bits.y, bits.z, bits.w};
  uint32_t of[4] = {off.x, off.y, off.z, off.w};
  int c = 0;
  while (c + 1 < n_chunks && idx >= of[c + 1]) ++c;
  uint32_t loc = idx - of[c];
  uint32_t a = loc >> bw[c], b = loc & ((1u << bw[c]) - 1u);
  double acc = 0.0;
  for (int i = 0; i < bw[c]; ++i)
    if (((a >> i) & 1u) && ((b >> i) & 1u)) acc += U[w_lo + 8 * c + i];
  if (c == oc)
    for (int x = o0; x < o0 + M; ++x)
      for (int y = o0; y < o0 + M; ++y)
        if (x != y && ((a >> x) & 1u) && ((b >> y) & 1u)) acc += Up;
  W[idx] = acc;
}

// Spin-flip / pair-hop list per up string.  For an ordered impurity pair (a, b)
// with a occupied and b empty in the row string u, the column string is
// u - a + b with one-body sign s_u; the spin-flip partner moves the down
// electron b -> a (column d - b + a), the pair-hop partner moves it a -> b.
// Matrix element: +J' s_u s_d (the Sec. 4 Hamiltonian's -J' with the two
// one-body bilinears reordered).
__global__ void k_mix_count(uint32_t D, int M, int o0, int nsf, int nph,
                            const uint32_t* __restrict__ basis, uint32_t* __restrict__ count) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D) return;
  uint32_t s = basis[r] >> o0;
  uint32_t c = 0;
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b)
      if (a != b && ((s >> a) & 1u) && !((s >> b) & 1u)) c += nsf + nph;
  count[r] = c;
}

__global__ void k_mix_fill(uint32_t D, int M, int o0, double Jsf, double Jph,
                           const uint32_t* __restrict__ basis, const uint32_t* __restrict__ C,
                           const uint32_t* __restrict__ ptr, uint32_t* __restrict__ tgt,
                           double* __restrict__ val, uint8_t* __restrict__ mv) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D) return;
  uint32_t s = basis[r];
  uint32_t o = ptr[r];
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      const int sa = o0 + a, sb = o0 + b;
      if (a == b || !((s >> sa) & 1u) || ((s >> sb) & 1u)) continue;
      uint32_t t = rank_of(s ^ (1u << sa) ^ (1u << sb), C);
      double su = (__popc(s & between(sa, sb)) & 1) ? -1.0 : 1.0;
      if (Jsf != 0.0) {
        tgt[o] = t;
        val[o] = Jsf * su;
        mv[o] = (uint8_t)(b * M + a);
        ++o;
      }
      if (Jph != 0.0) {
        tgt[o] = t;
        val[o] = Jph * su;
        mv[o] = (uint8_t)(a * M + b);
        ++o;
      }
    }
}

// Down-move tables: entry [x*M + y][d] = rank(d - x + y) << 1 | sign bit when
// x is occupied and y empty in d, else -1.
__global__ void k_move(uint32_t D, int M, int o0, const uint32_t* __restrict__ basis,
                       const uint32_t* __restrict__ C, int32_t* __restrict__ mv) {
  uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)D * M * M) return;
  uint32_t p = (uint32_t)(idx / D), d = (uint32_t)(idx % D);
  int x = o0 + (int)(p / M), y = o0 + (int)(p % M);
  uint32_t s = basis[d];
  int32_t out = -1;
  if (x != y && ((s >> x) & 1u) && !((s >> y) & 1u)) {
    uint32_t t = rank_of(s ^ (1u << x) ^ (1u << y), C);
    out = (int32_t)((t << 1) | (uint32_t)(__popc(s & between(x, y)) & 1));
  }
  mv[idx] = out;
}

__global__ void k_to_df(const double* __restrict__ a, float2* __restrict__ b, uint64_t n) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = df_from_double(a[i]);
}

// Map of each string of the target sector's changed spin to the source rank
// (or -1) and the Jordan-Wigner sign bit of c+ / c acting there.
__global__ void k_cop_map(uint32_t Dt, const uint32_t* __restrict__ tbasis, int orbital,
                          int dagger, const uint32_t* __restrict__ C, int32_t* __restrict__ map) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Dt) return;
  uint32_t t = tbasis[r];
  uint32_t bit = 1u << orbital;
  bool ok = dagger ? (t & bit) : !(t & bit);
  int32_t out = -1;
  if (ok) {
    uint32_t s = t ^ bit;
    uint32_t below = t & (bit - 1u);
    out = (int32_t)((rank_of(s, C) << 1) | (uint32_t)(__popc(below) & 1));
  }
  map[r] = out;
}

template <class V>
__device__ __forceinline__ V negate(V v);
template <>
__device__ __forceinline__ double negate<double>(double v) { return -v; }
template <>
__device__ __forceinline__ float negate<float>(float v) { return -v; }
template <>
__device__ __forceinline__ float2 negate<float2>(float2 v) { return make_float2(-v.x, -v.y); }
template <class V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ double vzero<double>() { return 0.0; }
template <>
__device__ __forceinline__ float vzero<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }

// phi[r_up', r_dn'] = sign * psi[r_up, r_dn] with one spin's rank mapped.
template <class V>
__global__ void k_cop_apply(const V* __restrict__ psi, V* __restrict__ phi, const int32_t* __restrict__ map,
                            int spin_dn, uint32_t Dtu, uint32_t Dtd, uint32_t Dsd, int extra_sign) {
  uint64_t n = (uint64_t)Dtu * Dtd;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u = (uint32_t)(i / Dtd), d = (uint32_t)(i % Dtd);
    int32_t m = map[spin_dn ? d : u];
    V out = vzero<V>();
    if (m >= 0) {
      uint32_t src = (uint32_t)(m >> 1);
      uint64_t j = spin_dn ? (uint64_t)u * Dsd + src : (uint64_t)src * Dsd + d;
      V v = psi[j];
      out = (((m & 1) ^ extra_sign) ? negate<V>(v) : v);
    }
    phi[i] = out;
  }
}

inline uint32_t nblk(uint64_t n, int bs) { return (uint32_t)((n + bs - 1) / bs); }

int host_scan(std::vector<uint32_t>& cnt, uint64_t* total) {
  uint64_t run = 0;
  for (size_t i = 0; i < cnt.size(); ++i) {
    uint64_t c = cnt[i];
    cnt[i] = (uint32_t)run;
    run += c;
    if (run > 0xffffffffull) ED_INVALID("table too large (%llu entries)", (unsigned long long)run);
  }
  *total = run;
  return ED_OK;
}

int build_spin(Sector* s, const double* dT, int n, SpinTables* sp) {
  Ctx* c = s->ctx;
  sp->n = n;
  uint64_t D = 1;
  {
    // C(n_s, n) from the host copy of the table
    uint64_t num = 1;
    for (int i = 0; i < n; ++i) num = num * (uint64_t)(s->n_s - i) / (uint64_t)(i + 1);
    D = num;
  }
  if (D > 0x7fffffffull) ED_INVALID("spin dimension %llu too large", (unsigned long long)D);
  sp->D = (uint32_t)D;
  ED_TRY(sector_alloc(s, &sp->basis, D));
  ED_TRY(sector_alloc(s, &sp->e, D));
  ED_TRY(sector_alloc(s, &sp->hop_ptr, D + 1));
  ModelArgs ma{s->n_s, s->M, s->orb0, s->Up - s->J, dT};
  k_spin_count<<<nblk(D, 128), 128>>>(ma, n, (uint32_t)D, c->d_binom, sp->basis, sp->e, sp->hop_ptr);
  ED_LAUNCH_CHECK();
  std::vector<uint32_t> cnt(D + 1, 0);
  ED_TRY_CUDA(cudaMemcpy(cnt.data(), sp->hop_ptr, D * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  sp->max_hops = D ? *std::max_element(cnt.begin(), cnt.begin() + D) : 0;
  if (sp->max_hops > (uint32_t)kMaxLocal) ED_INVALID("too many hops per string");
  ED_TRY(host_scan(cnt, &sp->n_hops));
  ED_TRY_CUDA(cudaMemcpy(sp->hop_ptr, cnt.data(), (D + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice));
  ED_TRY(sector_alloc(s, &sp->hop_tgt, sp->n_hops));
  ED_TRY(sector_alloc(s, &sp->hop_val, sp->n_hops));
  k_spin_fill<<<nblk(D, 64), 64>>>(ma, (uint32_t)D, c->d_binom, sp->basis, sp->hop_ptr, sp->hop_tgt,
                                   sp->hop_val);
  ED_LAUNCH_CHECK();
  if (s->prec != ED_PREC_FP64) {
    ED_TRY(sector_alloc(s, &sp->hop_val_df, sp->n_hops));
    ED_TRY(sector_alloc(s, &sp->e_df, D));
    if (sp->n_hops) k_to_df<<<nblk(sp->n_hops, 256), 256>>>(sp->hop_val, sp->hop_val_df, sp->n_hops);
    k_to_df<<<nblk(D, 256), 256>>>(sp->e, sp->e_df, D);
    ED_LAUNCH_CHECK();
  }
  return ED_OK;
}

}  // namespace

int validate_model(const ed_model* m) {
  if (!m || !m->T || !m->U_site) ED_INVALID("model or its arrays are NULL");
  if (m->n_s < 1 || m->n_s > ED_MAX_SITES) ED_INVALID("n_s=%d outside 1..%d", m->n_s, ED_MAX_SITES);
  if (m->n_orb < 0 || m->n_orb > ED_MAX_ORB || m->n_orb > m->n_s)
    ED_INVALID("n_orb=%d outside 0..min(n_s, %d)", m->n_orb, ED_MAX_ORB);
  if (m->orb0 < 0 || m->orb0 + m->n_orb > m->n_s)
    ED_INVALID("orbital sites %d..%d outside 0..%d", m->orb0, m->orb0 + m->n_orb - 1, m->n_s - 1);
  for (int i = 0; i < m->n_s; ++i)
    for (int j = 0; j < m->n_s; ++j) {
      double a = m->T[i * m->n_s + j], b = m->T[j * m->n_s + i];
      if (!std::isfinite(a)) ED_INVALID("T[%d][%d] not finite", i, j);
      if (a != b) ED_INVALID("T not symmetric at (%d,%d)", i, j);
    }
  for (int i = 0; i < m->n_s; ++i)
    if (!std::isfinite(m->U_site[i])) ED_INVALID("U_site[%d] not finite", i);
  if (!std::isfinite(m->Up) || !std::isfinite(m->J) || !std::isfinite(m->Jsf) || !std::isfinite(m->Jph))
    ED_INVALID("interaction constants not finite");
  return ED_OK;
}

SectorView Sector::view() const {
  SectorView v;
  v.D_up = up.D;
  v.D_dn = dn.D;
  v.n_s = n_s;
  v.M = M;
  v.w_lo = w_lo;
  v.n_chunks = n_chunks;
  for (int c = 0; c < 4; ++c) {
    v.w_bits[c] = w_bits[c];
    v.w_off[c] = w_off[c];
  }
  v.W = W;
  v.W_df = W_df;
  v.uh_ptr = up.hop_ptr;
  v.uh_tgt = up.hop_tgt;
  v.uh_val = up.hop_val;
  v.uh_val_df = up.hop_val_df;
  v.dh_ptr = dn.hop_ptr;
  v.dh_tgt = dn.hop_tgt;
  v.dh_val = dn.hop_val;
  v.dh_val_df = dn.hop_val_df;
  v.e_up = up.e;
  v.e_dn = dn.e;
  v.e_up_df = up.e_df;
  v.e_dn_df = dn.e_df;
  v.mx_ptr = mx_ptr;
  v.mx_tgt = mx_tgt;
  v.mx_val = mx_val;
  v.mx_val_df = mx_val_df;
  v.mx_mv = mx_mv;
  v.dn_move = dn_move;
  return v;
}

void free_sector(Sector* s) {
  for (auto& a : s->allocs) dev_free(s->ctx, a.first, a.second);
  s->allocs.clear();
  s->table_bytes = 0;
}

int build_sector(Ctx* ctx, const ed_model* m, int n_up, int n_dn, int prec, Sector* s) {
  ED_TRY(validate_model(m));
  if (n_up < 0 || n_up > m->n_s || n_dn < 0 || n_dn > m->n_s)
    ED_INVALID("particle numbers (%d,%d) outside 0..%d", n_up, n_dn, m->n_s);
  if (prec != ED_PREC_FP64 && prec != ED_PREC_DF64 && prec != ED_PREC_FP32)
    ED_INVALID("unknown precision %d", prec);
  s->ctx = ctx;
  s->n_s = m->n_s;
  s->n_up = n_up;
  s->n_dn = n_dn;
  s->prec = prec;
  s->M = m->n_orb;
  s->orb0 = m->orb0;
  std::memcpy(s->T, m->T, sizeof(double) * m->n_s * m->n_s);
  std::memcpy(s->U_site, m->U_site, sizeof(double) * m->n_s);
  s->Up = m->Up;
  s->J = m->J;
  s->Jsf = m->Jsf;
  s->Jph = m->Jph;
  ED_TRY_CUDA(cudaSetDevice(ctx->device));

  double* dT = nullptr;
  ED_TRY(sector_alloc(s, &dT, (size_t)s->n_s * s->n_s));
  ED_TRY_CUDA(cudaMemcpy(dT, s->T, sizeof(double) * s->n_s * s->n_s, cudaMemcpyHostToDevice));
  ED_TRY(build_spin(s, dT, n_up, &s->up));
  ED_TRY(build_spin(s, dT, n_dn, &s->dn));
  s->dim = (uint64_t)s->up.D * s->dn.D;

  // cross tables over the window of sites carrying U_site or an orbital
  int lo = s->n_s, hi = 0;
  if (s->M > 0) {
    lo = s->orb0;
    hi = s->orb0 + s->M;
  }
  for (int i = 0; i < s->n_s; ++i)
    if (s->U_site[i] != 0.0) {
      lo = std::min(lo, i);
      hi = std::max(hi, i + 1);
    }
  int K = hi > lo ? hi - lo : 0;
  s->w_lo = K ? lo : 0;
  s->K = K;
  s->n_chunks = (K + 7) / 8;
  int ocnk = 0, obit = 0;
  if (s->M > 0) {
    ocnk = (s->orb0 - s->w_lo) / 8;
    obit = (s->orb0 - s->w_lo) % 8;
    if ((s->orb0 + s->M - 1 - s->w_lo) / 8 != ocnk)
      ED_INVALID("impurity orbitals straddle an 8-site block of the interaction window");
  }
  uint32_t total = 0;
  for (int c = 0; c < s->n_chunks; ++c) {
    s->w_bits[c] = std::min(8, K - 8 * c);
    s->w_off[c] = total;
    total += 1u << (2 * s->w_bits[c]);
  }
  s->w_size = total;
  if (total) {
    double* dU = nullptr;
    ED_TRY(sector_alloc(s, &dU, 32));
    double Upad[32] = {0};
    std::memcpy(Upad, s->U_site, sizeof(double) * s->n_s);
    ED_TRY_CUDA(cudaMemcpy(dU, Upad, sizeof(Upad), cudaMemcpyHostToDevice));
    ED_TRY(sector_alloc(s, &s->W, total));
    k_cross<<<nblk(total, 256), 256>>>(s->n_chunks,
                                       make_int4(s->w_bits[0], s->w_bits[1], s->w_bits[2], s->w_bits[3]),
                                       make_uint4(s->w_off[0], s->w_off[1], s->w_off[2], s->w_off[3]),
                                       dU, s->w_lo, s->M, ocnk, obit, s->Up, total, s->W);
    ED_LAUNCH_CHECK();
    if (prec != ED_PREC_FP64) {
      ED_TRY(sector_alloc(s, &s->W_df, total));
      k_to_df<<<nblk(total, 256), 256>>>(s->W, s->W_df, total);
      ED_LAUNCH_CHECK();
    }
  }

  // spin-flip / pair-hop
  int nsf = (s->Jsf != 0.0), nph = (s->Jph != 0.0);
  if (s->M >= 2 && (nsf || nph)) {
    uint32_t D = s->up.D;
    ED_TRY(sector_alloc(s, &s->mx_ptr, (size_t)D + 1));
    k_mix_count<<<nblk(D, 128), 128>>>(D, s->M, s->orb0, nsf, nph, s->up.basis, s->mx_ptr);
    ED_LAUNCH_CHECK();
    std::vector<uint32_t> cnt(D + 1, 0);
    ED_TRY_CUDA(cudaMemcpy(cnt.data(), s->mx_ptr, D * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    s->max_mix = D ? *std::max_element(cnt.begin(), cnt.begin() + D) : 0;
    ED_TRY(host_scan(cnt, &s->n_mix));
    ED_TRY_CUDA(cudaMemcpy(s->mx_ptr, cnt.data(), (D + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice));
    ED_TRY(sector_alloc(s, &s->mx_tgt, s->n_mix));
    ED_TRY(sector_alloc(s, &s->mx_val, s->n_mix));
    ED_TRY(sector_alloc(s, &s->mx_mv, s->n_mix));
    k_mix_fill<<<nblk(D, 128), 128>>>(D, s->M, s->orb0, s->Jsf, s->Jph, s->up.basis, ctx->d_binom, s->mx_ptr,
                                      s->mx_tgt, s->mx_val, s->mx_mv);
    ED_LAUNCH_CHECK();
    uint64_t nm = (uint64_t)s->dn.D * s->M * s->M;
    ED_TRY(sector_alloc(s, &s->dn_move, nm));
    k_move<<<nblk(nm, 256), 256>>>(s->dn.D, s->M, s->orb0, s->dn.basis, ctx->d_binom, s->dn_move);
    ED_LAUNCH_CHECK();
    if (prec != ED_PREC_FP64 && s->n_mix) {
      ED_TRY(sector_alloc(s, &s->mx_val_df, s->n_mix));
      k_to_df<<<nblk(s->n_mix, 256), 256>>>(s->mx_val, s->mx_val_df, s->n_mix);
      ED_LAUNCH_CHECK();
    }
  }
  ED_TRY_CUDA(cudaStreamSynchronize(0));  // legacy stream only: leaves other work running
  return ED_OK;
}

// ------------------------------------------------------------- c+ / c maps
int apply_cop(const Sector* src, const Sector* dst, int orbital, int spin, bool dagger,
              const void* psi, void* phi, cudaStream_t st) {
  if (src->prec != dst->prec) ED_INVALID("sector precisions differ");
  if (orbital < 0 || orbital >= src->n_s) ED_INVALID("orbital %d outside 0..%d", orbital, src->n_s - 1);
  int du = (spin == ED_SPIN_UP) ? (dagger ? 1 : -1) : 0;
  int dd = (spin == ED_SPIN_DN) ? (dagger ? 1 : -1) : 0;
  if (dst->n_up != src->n_up + du || dst->n_dn != src->n_dn + dd || dst->n_s != src->n_s)
    ED_INVALID("target sector does not match the operator");
  const SpinTables& tsp = (spin == ED_SPIN_UP) ? dst->up : dst->dn;
  int32_t* map = nullptr;
  Sector* mut = const_cast<Sector*>(dst);
  // one map per call; freed with the call's temporary below
  ED_TRY(dev_alloc_n(dst->ctx, &map, (size_t)tsp.D + 1));
  k_cop_map<<<nblk(tsp.D, 128), 128, 0, st>>>(tsp.D, tsp.basis, orbital, dagger ? 1 : 0,
                                              dst->ctx->d_binom, map);
  // c+ / c for a down electron also passes every up electron: (-1)^{N_up}
  int extra = (spin == ED_SPIN_DN) ? (src->n_up & 1) : 0;
  int sdn = (spin == ED_SPIN_DN) ? 1 : 0;
  uint32_t grid = (uint32_t)std::min<uint64_t>(nblk(dst->dim, 256), 65535u * 4);
  if (grid == 0) grid = 1;
  switch (src->prec) {
    case ED_PREC_FP64:
      k_cop_apply<double><<<grid, 256, 0, st>>>((const double*)psi, (double*)phi, map, sdn, dst->up.D,
                                                dst->dn.D, src->dn.D, extra);
      break;
    case ED_PREC_DF64:
      k_cop_apply<float2><<<grid, 256, 0, st>>>((const float2*)psi, (float2*)phi, map, sdn, dst->up.D,
                                                dst->dn.D, src->dn.D, extra);
      break;
    default:
      k_cop_apply<float><<<grid, 256, 0, st>>>((const float*)psi, (float*)phi, map, sdn, dst->up.D,
                                               dst->dn.D, src->dn.D, extra);
  }
  cudaError_t e = cudaGetLastError();
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  dev_free(dst->ctx, map, ((size_t)tsp.D + 1) * sizeof(int32_t));
  (void)mut;
  if (e != cudaSuccess) {
    set_error("c+/c map launch failed: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  return ED_OK;
}

}  // namespace ed
