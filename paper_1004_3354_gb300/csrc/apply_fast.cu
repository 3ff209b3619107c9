// Row kernel for the matrix-free H*v on long rows (the production path).
//
// Same operator as apply.cu (one-body hops of both spins, the diagonal of
// Eq. 1 / Eq. 2 / the Sec. 4 Hamiltonian, spin-flip and pair-hopping), laid
// out for the GPU:
//
//  * Rows (up strings) are visited in an order that groups the connected
//    components of the up-spin one-body hop graph (strings with equal electron
//    counts on each bond-connected cluster of sites), so the x rows that the
//    up hops of concurrently processed rows read stay resident in L2.
//  * Each block stages one x row in shared memory and runs two passes over it:
//    pass 1 walks the row in a fixed permutation of the down strings sorted by
//    (diagonal pattern, hop count), so every warp executes the same number of
//    down hops and the same spin-flip / pair-hop branches; it accumulates the
//    down hops, the down part of the diagonal and the spin-flip / pair-hop
//    terms into a shared-memory accumulator row.  Pass 2 walks the row in
//    natural order, adds the up-spin part of the diagonal and the up hops
//    (coalesced reads of neighbouring x rows) and writes y once.
//  * Down-hop entries are packed 4-byte words (target rank << 8 | coefficient
//    id) with the distinct matrix elements held in shared memory.
#include <algorithm>
#include <functional>
#include <map>
#include <numeric>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr int kList = 128;      // max up hops / mixed entries per row on the fast path
constexpr int kMaxCoef = 256;

struct FastView {
  uint32_t D_up, D, D4;
  const uint32_t* row_order;
  const uint32_t* row_pat;
  const uint4* perm4;           // [D4/4] q -> d, four at a time
  const uint8_t* cnt4;          // [D4/4] widest hop list among four consecutive q
  const uint4* hop4;            // [max_cnt][D4/4] packed hop words
  const double* coef;
  const float2* coef_df;
  int n_coef;
  const double* dd;             // [n_pat][D4]
  const float2* dd_df;
  const int32_t* mv;            // natural-order down-move tables [M*M][D]
  const uint32_t *uh_ptr, *uh_tgt;
  const double* uh_val;
  const float2* uh_val_df;
  const double* e_up;
  const float2* e_up_df;
  const uint32_t *mx_ptr, *mx_tgt;
  const double* mx_val;
  const float2* mx_val_df;
  const uint8_t* mx_mv;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <class P>
size_t fast_smem(uint32_t D, int n_coef) {
  using V = typename P::V;
  using A = typename P::A;
  using C = typename P::C;
  return align16(D * sizeof(V)) + align16(D * sizeof(A)) + align16(n_coef * sizeof(C)) +
         2 * align16(kList * sizeof(C)) + 2 * align16(kList * sizeof(uint64_t)) + align16(kList * 4);
}

// four diagonal-table entries for consecutive q (16-byte aligned groups)
template <class C>
__device__ __forceinline__ void ld4(const C* p, C (&o)[4]);
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double (&o)[4]) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <>
__device__ __forceinline__ void ld4<float2>(const float2* p, float2 (&o)[4]) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  o[0] = make_float2(a.x, a.y); o[1] = make_float2(a.z, a.w);
  o[2] = make_float2(b.x, b.y); o[3] = make_float2(b.z, b.w);
}

template <class V>
__device__ __forceinline__ void st_stream(V* p, V v) { __stcs(p, v); }

template <class P, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_apply_fast(FastView F, const typename P::V* __restrict__ x,
                                                        typename P::V* __restrict__ y) {
  using V = typename P::V;
  using A = typename P::A;
  using C = typename P::C;
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t D = F.D, G4 = F.D4 >> 2;
  unsigned char* p = sm;
  V* xs = reinterpret_cast<V*>(p);
  p += align16(D * sizeof(V));
  A* ys = reinterpret_cast<A*>(p);
  p += align16(D * sizeof(A));
  C* cs = reinterpret_cast<C*>(p);
  p += align16(F.n_coef * sizeof(C));
  C* lc = reinterpret_cast<C*>(p);          // up-hop coefficients
  p += align16(kList * sizeof(C));
  C* mc = reinterpret_cast<C*>(p);          // mixed coefficients
  p += align16(kList * sizeof(C));
  uint64_t* lr = reinterpret_cast<uint64_t*>(p);  // up-hop row offsets (elements)
  p += align16(kList * sizeof(uint64_t));
  uint64_t* mr = reinterpret_cast<uint64_t*>(p);  // mixed row offsets
  p += align16(kList * sizeof(uint64_t));
  uint32_t* mm = reinterpret_cast<uint32_t*>(p);  // mixed move-table offsets
  __shared__ int n_up_s, n_mx_s;
  __shared__ uint32_t pat_s;

  for (int k = threadIdx.x; k < F.n_coef; k += BS) cs[k] = P::ld(F.coef, F.coef_df, k);

  for (uint32_t i = blockIdx.x; i < F.D_up; i += gridDim.x) {
    const uint32_t u = F.row_order[i];
    __syncthreads();
    const V* xr = x + (uint64_t)u * D;
    for (uint32_t d = threadIdx.x; d < D; d += BS) xs[d] = xr[d];
    const uint32_t h0 = F.uh_ptr[u], nh = F.uh_ptr[u + 1] - h0;
    for (uint32_t k = threadIdx.x; k < nh; k += BS) {
      lr[k] = (uint64_t)F.uh_tgt[h0 + k] * D;
      lc[k] = P::ld(F.uh_val, F.uh_val_df, h0 + k);
    }
    uint32_t nm = 0;
    if (F.mx_ptr) {
      const uint32_t m0 = F.mx_ptr[u];
      nm = F.mx_ptr[u + 1] - m0;
      for (uint32_t k = threadIdx.x; k < nm; k += BS) {
        mr[k] = (uint64_t)F.mx_tgt[m0 + k] * D;
        mc[k] = P::ld(F.mx_val, F.mx_val_df, m0 + k);
        mm[k] = (uint32_t)F.mx_mv[m0 + k] * D;
      }
    }
    if (threadIdx.x == 0) {
      n_up_s = (int)nh;
      n_mx_s = (int)nm;
      pat_s = F.row_pat[u];
    }
    __syncthreads();
    // pass 1, permuted order, four consecutive q per thread: the down part of
    // the diagonal and the down hops (hop counts equal within a warp)
    {
      const C* ddr = P::ld_ptr(F.dd, F.dd_df) + (uint64_t)pat_s * F.D4;
      for (uint32_t g = threadIdx.x; g < G4; g += BS) {
        const uint4 pp = F.perm4[g];
        const uint32_t pv[4] = {pp.x, pp.y, pp.z, pp.w};
        C dg[4];
        ld4<C>(ddr + 4 * (uint64_t)g, dg);
        A acc[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc[e] = P::zero();
          P::mac(acc[e], dg[e], xs[pv[e]]);
        }
        const int c = F.cnt4[g];
        const uint4* hp = F.hop4 + g;
        for (int k = 0; k < c; ++k) {
          const uint4 w = __ldg(hp + (uint64_t)k * G4);
          const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) P::mac(acc[e], cs[wv[e] & 255u], xs[wv[e] >> 8]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (4 * g + e < D) ys[pv[e]] = acc[e];
      }
    }
    __syncthreads();
    // pass 2, natural order, four strided elements per thread: the up part of
    // the diagonal, the up hops, spin-flip / pair-hop, one store
    {
      const C eu = P::ld(F.e_up, F.e_up_df, u);
      const int nup = n_up_s, nmx = n_mx_s;
      V* yr = y + (uint64_t)u * D;
      for (uint32_t d0 = threadIdx.x; d0 < D; d0 += 4 * BS) {
        uint32_t dv[4];
        bool ok[4];
        A acc[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          dv[e] = d0 + e * BS;
          ok[e] = dv[e] < D;
          const uint32_t dd = ok[e] ? dv[e] : d0;
          acc[e] = ys[dd];
          P::mac(acc[e], eu, xs[dd]);
        }
        for (int k = 0; k < nup; ++k) {
          const C c = lc[k];
          const V* xk = x + lr[k];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (ok[e]) P::mac(acc[e], c, __ldg(xk + dv[e]));
        }
        for (int j = 0; j < nmx; ++j) {
          const int32_t* mvt = F.mv + mm[j];
          const V* xm = x + mr[j];
          const C cj = mc[j];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (!ok[e]) continue;
            const int32_t mvv = __ldg(mvt + dv[e]);
            if (mvv >= 0) P::mac(acc[e], (mvv & 1) ? P::neg(cj) : cj, __ldg(xm + (uint32_t)(mvv >> 1)));
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (ok[e]) st_stream(yr + dv[e], P::out(acc[e]));
      }
    }
  }
}

// Permuted per-down-string tables, padded to D4 = 4 * ceil(D / 4) entries.
__global__ void k_fast_tables(uint32_t D, uint32_t D4, const uint32_t* __restrict__ perm,
                              const uint32_t* __restrict__ dbasis, const uint32_t* __restrict__ dh_ptr,
                              const uint32_t* __restrict__ dh_tgt, const double* __restrict__ dh_val,
                              const double* __restrict__ coef, int n_coef, int zero_id, uint32_t max_cnt,
                              uint32_t* __restrict__ perm_out, uint8_t* __restrict__ cnt4,
                              uint32_t* __restrict__ hop, const double* __restrict__ e_dn,
                              const double* __restrict__ W, int w_lo, int wbits, int n_pat,
                              double* __restrict__ dd) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= D4) return;
  const bool real = q < D;
  const uint32_t d = real ? perm[q] : 0u;
  const uint32_t h0 = dh_ptr[d], c = real ? dh_ptr[d + 1] - h0 : 0u;
  perm_out[q] = d;
  for (uint32_t k = 0; k < max_cnt; ++k) {
    uint32_t word = (uint32_t)zero_id;  // target 0 times a zero coefficient
    if (k < c) {
      double v = dh_val[h0 + k];
      int id = 0;
      while (id < n_coef && coef[id] != v) ++id;
      word = (dh_tgt[h0 + k] << 8) | (uint32_t)(id & 255);
    }
    hop[(uint64_t)k * D4 + q] = word;
  }
  // widest list among the four q of this group
  if ((q & 3u) == 0) {
    uint32_t c4 = 0;
    for (uint32_t e = 0; e < 4 && q + e < D; ++e) {
      const uint32_t de = perm[q + e];
      c4 = max(c4, dh_ptr[de + 1] - dh_ptr[de]);
    }
    cnt4[q >> 2] = (uint8_t)c4;
  }
  const uint32_t pd = (wbits > 0) ? ((dbasis[d] >> w_lo) & ((1u << wbits) - 1u)) : 0u;
  for (int pu = 0; pu < n_pat; ++pu) {
    double v = real ? e_dn[d] : 0.0;
    if (W && real) v += W[((uint32_t)pu << wbits) + pd];
    dd[(uint64_t)pu * D4 + q] = v;
  }
}

__global__ void k_row_pat(uint32_t D, const uint32_t* __restrict__ ub, int w_lo, int wbits,
                          uint32_t* __restrict__ pat) {
  uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < D) pat[u] = (wbits > 0) ? ((ub[u] >> w_lo) & ((1u << wbits) - 1u)) : 0u;
}

__global__ void k_df_copy(const double* __restrict__ a, float2* __restrict__ b, uint64_t n) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = df_from_double(a[i]);
}

template <class P>
FastView make_view(const Sector* s) {
  FastView F;
  const auto& f = s->fast;
  F.D_up = s->up.D;
  F.D = s->dn.D;
  F.D4 = (F.D + 3u) & ~3u;
  F.row_order = f.row_order;
  F.row_pat = f.row_pat;
  F.perm4 = reinterpret_cast<const uint4*>(f.perm);
  F.cnt4 = f.cnt;
  F.hop4 = reinterpret_cast<const uint4*>(f.hop);
  F.coef = f.coef;
  F.coef_df = f.coef_df;
  F.n_coef = f.n_coef;
  F.dd = f.dd;
  F.dd_df = f.dd_df;
  F.mv = s->dn_move;
  F.uh_ptr = s->up.hop_ptr;
  F.uh_tgt = s->up.hop_tgt;
  F.uh_val = s->up.hop_val;
  F.uh_val_df = s->up.hop_val_df;
  F.e_up = s->up.e;
  F.e_up_df = s->up.e_df;
  F.mx_ptr = s->mx_ptr;
  F.mx_tgt = s->mx_tgt;
  F.mx_val = s->mx_val;
  F.mx_val_df = s->mx_val_df;
  F.mx_mv = s->mx_mv;
  return F;
}

template <class P, int BS, int MINB>
int launch_fast(const Sector* s, const void* x, void* y, cudaStream_t st) {
  FastView F = make_view<P>(s);
  size_t smem = fast_smem<P>(F.D, F.n_coef);
  auto kern = k_apply_fast<P, BS, MINB>;
  ED_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem));
  if (per_sm < 1) ED_INVALID("fast row kernel does not fit on an SM (%zu B shared)", smem);
  uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)s->ctx->num_sms * per_sm, F.D_up);
  kern<<<grid, BS, smem, st>>>(F, static_cast<const typename P::V*>(x), static_cast<typename P::V*>(y));
  ED_LAUNCH_CHECK();
  return ED_OK;
}

template <class P>
int dispatch(const Sector* s, const void* x, void* y, cudaStream_t st) {
  size_t smem = fast_smem<P>(s->dn.D, s->fast.n_coef);
  if (smem <= 110 * 1024) return launch_fast<P, 512, 2>(s, x, y, st);
  return launch_fast<P, 1024, 1>(s, x, y, st);
}

}  // namespace

int build_fast(Sector* s) {
  s->fast.ok = false;
  const uint32_t D = s->dn.D;
  if (D < 1024 || s->n_chunks > 1 || s->up.max_hops > (uint32_t)kList || s->max_mix > (uint32_t)kList)
    return ED_OK;
  if (s->dn.max_hops > 64 || D >= (1u << 24)) return ED_OK;
  // distinct down-hop matrix elements
  std::vector<double> hv(s->dn.n_hops);
  if (s->dn.n_hops)
    ED_TRY_CUDA(cudaMemcpy(hv.data(), s->dn.hop_val, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost));
  std::vector<double> coef;
  {
    std::map<double, int> seen;
    for (double v : hv)
      if (!seen.count(v)) {
        seen[v] = (int)coef.size();
        coef.push_back(v);
        if (coef.size() > (size_t)kMaxCoef) return ED_OK;
      }
  }
  if (coef.empty()) coef.push_back(0.0);
  size_t smem_max = std::max(fast_smem<PolF64>(D, (int)coef.size()), fast_smem<PolDF>(D, (int)coef.size()));
  if (smem_max > 220 * 1024) return ED_OK;

  // permutation of the down strings: sort by (diagonal pattern, hop count, rank)
  const int wbits = (s->n_chunks == 1) ? s->w_bits[0] : 0;
  std::vector<uint32_t> dbas(D), dptr(D + 1);
  ED_TRY_CUDA(cudaMemcpy(dbas.data(), s->dn.basis, sizeof(uint32_t) * D, cudaMemcpyDeviceToHost));
  ED_TRY_CUDA(cudaMemcpy(dptr.data(), s->dn.hop_ptr, sizeof(uint32_t) * (D + 1), cudaMemcpyDeviceToHost));
  std::vector<uint32_t> perm(D);
  std::iota(perm.begin(), perm.end(), 0u);
  auto key = [&](uint32_t d) {
    uint32_t pd = wbits ? ((dbas[d] >> s->w_lo) & ((1u << wbits) - 1u)) : 0u;
    return ((uint64_t)pd << 32) | (uint64_t)(dptr[d + 1] - dptr[d]);
  };
  std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return key(a) < key(b); });

  // row order: group up strings by electron counts on each bond-connected site cluster
  const int ns = s->n_s;
  std::vector<int> parent(ns);
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int(int)> find = [&](int a) { return parent[a] == a ? a : parent[a] = find(parent[a]); };
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j)
      if (i != j && s->T[i * ns + j] != 0.0) parent[find(i)] = find(j);
  std::vector<uint32_t> cmask;
  {
    std::map<int, uint32_t> m;
    for (int i = 0; i < ns; ++i) m[find(i)] |= 1u << i;
    for (auto& kv : m) cmask.push_back(kv.second);
  }
  const uint32_t Du = s->up.D;
  std::vector<uint32_t> ubas(Du), rorder(Du);
  ED_TRY_CUDA(cudaMemcpy(ubas.data(), s->up.basis, sizeof(uint32_t) * Du, cudaMemcpyDeviceToHost));
  std::vector<uint64_t> rkey(Du, 0);
  for (uint32_t u = 0; u < Du; ++u) {
    uint64_t k = 0;
    for (uint32_t mk : cmask) k = k * 33 + (uint64_t)__builtin_popcount(ubas[u] & mk);
    rkey[u] = cmask.size() <= 12 ? k : 0;
  }
  std::iota(rorder.begin(), rorder.end(), 0u);
  std::stable_sort(rorder.begin(), rorder.end(), [&](uint32_t a, uint32_t b) { return rkey[a] < rkey[b]; });

  auto& f = s->fast;
  f.max_cnt = s->dn.max_hops;
  // a zero coefficient pads the hop lists of groups whose four strings differ in length
  int zero_id = -1;
  for (size_t i = 0; i < coef.size(); ++i)
    if (coef[i] == 0.0) zero_id = (int)i;
  if (zero_id < 0) {
    if (coef.size() >= (size_t)kMaxCoef) return ED_OK;
    zero_id = (int)coef.size();
    coef.push_back(0.0);
  }
  f.n_coef = (int)coef.size();
  f.n_pat = 1 << wbits;
  const uint32_t D4 = (D + 3u) & ~3u;
  uint32_t* dperm = nullptr;
  ED_TRY(sector_alloc(s, &dperm, D));
  ED_TRY(sector_alloc(s, &f.perm, D4));
  ED_TRY(sector_alloc(s, &f.cnt, D4 / 4));
  ED_TRY(sector_alloc(s, &f.hop, (size_t)std::max(1u, f.max_cnt) * D4));
  ED_TRY(sector_alloc(s, &f.coef, f.n_coef));
  ED_TRY(sector_alloc(s, &f.dd, (size_t)f.n_pat * D4));
  ED_TRY(sector_alloc(s, &f.row_order, Du));
  ED_TRY(sector_alloc(s, &f.row_pat, Du));
  ED_TRY_CUDA(cudaMemcpy(dperm, perm.data(), sizeof(uint32_t) * D, cudaMemcpyHostToDevice));
  ED_TRY_CUDA(cudaMemcpy(f.coef, coef.data(), sizeof(double) * f.n_coef, cudaMemcpyHostToDevice));
  ED_TRY_CUDA(cudaMemcpy(f.row_order, rorder.data(), sizeof(uint32_t) * Du, cudaMemcpyHostToDevice));
  k_fast_tables<<<(D4 + 127) / 128, 128>>>(D, D4, dperm, s->dn.basis, s->dn.hop_ptr, s->dn.hop_tgt,
                                           s->dn.hop_val, f.coef, f.n_coef, zero_id, f.max_cnt, f.perm, f.cnt,
                                           f.hop, s->dn.e, (s->n_chunks == 1) ? s->W : nullptr, s->w_lo, wbits,
                                           f.n_pat, f.dd);
  ED_LAUNCH_CHECK();
  k_row_pat<<<(Du + 127) / 128, 128>>>(Du, s->up.basis, s->w_lo, wbits, f.row_pat);
  ED_LAUNCH_CHECK();
  if (s->prec != ED_PREC_FP64) {
    ED_TRY(sector_alloc(s, &f.coef_df, f.n_coef));
    ED_TRY(sector_alloc(s, &f.dd_df, (size_t)f.n_pat * D4));
    k_df_copy<<<(f.n_coef + 127) / 128, 128>>>(f.coef, f.coef_df, f.n_coef);
    k_df_copy<<<(unsigned)(((uint64_t)f.n_pat * D4 + 255) / 256), 256>>>(f.dd, f.dd_df, (uint64_t)f.n_pat * D4);
    ED_LAUNCH_CHECK();
  }
  ED_TRY_CUDA(cudaDeviceSynchronize());
  f.ok = true;
  return ED_OK;
}

int apply_fast(const Sector* s, const void* x, void* y, cudaStream_t st) {
  switch (s->prec) {
    case ED_PREC_FP64: return dispatch<PolF64>(s, x, y, st);
    case ED_PREC_DF64: return dispatch<PolDF>(s, x, y, st);
    case ED_PREC_FP32: return dispatch<PolF32>(s, x, y, st);
  }
  ED_INVALID("unknown precision");
}

}  // namespace ed
