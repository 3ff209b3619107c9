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
//  * A block stages one x row in shared memory (cp.async) and its warps sweep
//    the row in windows of 128 consecutive down strings.  Inside a window the
//    strings are sorted by hop count and dealt to 32 lanes x 4 slots, so the
//    lanes of a warp run the same number of down hops per slot, every global
//    access of the warp stays inside the window's 128 elements, and each thread
//    keeps its four elements in registers from the diagonal to the store.
//  * Down-hop entries are packed words holding the shared-memory byte offsets
//    of the target element (<< 13) and of its matrix element (the distinct
//    values live in shared memory); shorter lists in a slot are padded with
//    the zero coefficient.
//  * With the impurity orbitals on the top sites, down strings come in blocks
//    of equal impurity pattern and a spin-flip / pair-hop move shifts the rank
//    by a per-pattern constant, read from a small shared table.  At the start
//    of a row one warp builds, per impurity pattern, a term list: the row's up
//    hops followed by the spin-flip / pair-hop entries that apply to that
//    pattern, with the shift folded into the offset and the sign into the
//    coefficient.  A window whose strings share one pattern (most of them)
//    then gathers all its global terms in one loop, two at a time.
#include <algorithm>
#include <climits>
#include <functional>
#include <map>
#include <numeric>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr int kList = 64;       // max up hops / mixed entries per row on the fast path
constexpr int kMaxCoef = 256;
constexpr int kMaxDelta = 256;  // M*M*2^M entries of the move-shift table
constexpr int kWin = 128;       // strings per window = 32 lanes x 4 slots

struct FastView {
  uint32_t D_up, D, n_win, max_cnt;
  const uint32_t* row_order;
  const uint32_t* row_pat;
  const uint4* perm4;           // [n_win*32] four entries per lane
  const uchar4* cnt4;           // [n_win] slot counts
  const uint4* hop4;            // [n_win][max_cnt][32] (single-row or two-row encoding, per kernel)
  const double* coef;
  const float2* coef_df;
  int n_coef;
  const double* dd;             // [n_pat][n_win*128]
  const float2* dd_df;
  const int32_t* mv;            // natural-order down-move tables [M*M][D]
  const uint32_t* dpat4;        // [n_win*32] four impurity patterns per lane (delta layout) or NULL
  const uint32_t* wpat;         // [n_win] impurity pattern shared by the whole window, or ~0u
  const int32_t* mdelta;        // [M*M][np]
  int np, n_md;
  const uint32_t *uh_ptr, *uh_tgt;
  const double* uh_val;
  const float2* uh_val_df;
  const double* e_up;
  const float2* e_up_df;
  const uint32_t *mx_ptr, *mx_tgt;
  const double* mx_val;
  const float2* mx_val_df;
  const uint8_t* mx_mv;
  int n_lp;                     // term lists per row: 2^M with the delta layout, else 1
  uint32_t lcap;                // capacity of one list: longest up-hop plus spin-flip / pair-hop list
  double* dotp;                 // optional: per-block partial sums of <x, y>
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <class P>
size_t fast_smem(uint32_t D, int n_coef, int n_lp, uint32_t lcap) {
  using V = typename P::V;
  using C = typename P::C;
  const size_t nl = (size_t)n_lp * lcap;
  return align16(D * sizeof(V)) + align16(n_coef * sizeof(C)) + align16(nl * sizeof(C)) + align16(kList * sizeof(C)) +
         align16(nl * sizeof(int64_t)) + align16(kList * sizeof(uint64_t)) + align16(kList * 4) +
         align16(kMaxDelta * 4) + align16((size_t)n_lp * 4);
}

// four consecutive table entries (16-byte aligned)
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

// Asynchronous global -> shared copy of one element (cp.async, 4 or 8 bytes).
template <class V>
__device__ __forceinline__ void cp_async_elem(V* s, const V* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(g), "n"(sizeof(V)));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t sel4(const uint4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

template <class P, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_apply_win(FastView F, const typename P::V* __restrict__ x,
                                                       typename P::V* __restrict__ y) {
  using V = typename P::V;
  using A = typename P::A;
  using C = typename P::C;
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t D = F.D;
  unsigned char* p = sm;
  V* xs = reinterpret_cast<V*>(p);
  p += align16(D * sizeof(V));
  C* cs = reinterpret_cast<C*>(p);
  p += align16(F.n_coef * sizeof(C));
  const uint32_t lcap = F.lcap;
  const size_t nl = (size_t)F.n_lp * lcap;
  // term lists of the row, one per impurity pattern p (a single list without
  // the delta layout): the up hops, then the spin-flip / pair-hop entries that
  // apply to every down string of pattern p, with the pattern's rank shift
  // folded into the offset and its sign into the coefficient
  C* lc = reinterpret_cast<C*>(p);
  p += align16(nl * sizeof(C));
  C* mc = reinterpret_cast<C*>(p);          // mixed coefficients
  p += align16(kList * sizeof(C));
  int64_t* lr = reinterpret_cast<int64_t*>(p);    // element offsets of the list terms
  p += align16(nl * sizeof(int64_t));
  uint64_t* mr = reinterpret_cast<uint64_t*>(p);  // mixed row offsets
  p += align16(kList * sizeof(uint64_t));
  uint32_t* mm = reinterpret_cast<uint32_t*>(p);  // mixed move offsets
  p += align16(kList * 4);
  int32_t* mds = reinterpret_cast<int32_t*>(p);   // move shifts per pattern
  p += align16(kMaxDelta * 4);
  int* ln = reinterpret_cast<int*>(p);            // list lengths
  __shared__ int n_up_s, n_mx_s;
  __shared__ uint32_t pat_s;
  const bool mixd = F.dpat4 != nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NWARP = BS / 32;
  const uint64_t NE = (uint64_t)F.n_win * kWin;

  for (int k = threadIdx.x; k < F.n_coef; k += BS) cs[k] = P::ld(F.coef, F.coef_df, k);
  for (int k = threadIdx.x; k < F.n_md; k += BS) mds[k] = F.mdelta[k];
  A dacc = P::zero();  // <x, y> over this thread's elements (only used with F.dotp)

  for (uint32_t i = blockIdx.x; i < F.D_up; i += gridDim.x) {
    const uint32_t u = F.row_order[i];
    __syncthreads();
    const V* xr = x + (uint64_t)u * D;
    for (uint32_t d = threadIdx.x; d < D; d += BS) cp_async_elem(xs + d, xr + d);
    const uint32_t h0 = F.uh_ptr[u], nh = F.uh_ptr[u + 1] - h0;
    for (uint32_t k = threadIdx.x; k < nh; k += BS) {
      const int64_t off = (int64_t)F.uh_tgt[h0 + k] * D;
      const C c = P::ld(F.uh_val, F.uh_val_df, h0 + k);
      for (int q = 0; q < F.n_lp; ++q) {
        lr[q * lcap + k] = off;
        lc[q * lcap + k] = c;
      }
    }
    if (mixd && warp == NWARP - 1) {
      // list q gets, after the up hops and in entry order, the row's spin-flip /
      // pair-hop entries (at most kList = 64) that apply to impurity pattern q
      const uint32_t m0 = F.mx_ptr[u], nmr = F.mx_ptr[u + 1] - m0;
      const uint32_t ja = lane, jb = lane + 32;
      const bool va = ja < nmr, vb = jb < nmr;
      const int64_t ta = va ? (int64_t)F.mx_tgt[m0 + ja] * D : 0;
      const int64_t tb = vb ? (int64_t)F.mx_tgt[m0 + jb] * D : 0;
      const C ca = va ? P::ld(F.mx_val, F.mx_val_df, m0 + ja) : C{};
      const C cb = vb ? P::ld(F.mx_val, F.mx_val_df, m0 + jb) : C{};
      const uint32_t qa = va ? (uint32_t)F.mx_mv[m0 + ja] * (uint32_t)F.np : 0u;
      const uint32_t qb = vb ? (uint32_t)F.mx_mv[m0 + jb] * (uint32_t)F.np : 0u;
      const uint32_t below = (1u << lane) - 1u;
      for (int q = 0; q < F.n_lp; ++q) {
        const int32_t mda = va ? mds[qa + q] : INT_MIN, mdb = vb ? mds[qb + q] : INT_MIN;
        const unsigned ba = __ballot_sync(0xffffffffu, mda != INT_MIN);
        const unsigned bb = __ballot_sync(0xffffffffu, mdb != INT_MIN);
        const uint32_t base = q * lcap + nh;
        if (mda != INT_MIN) {
          const uint32_t at = base + __popc(ba & below);
          lr[at] = ta + (mda >> 1);
          lc[at] = (mda & 1) ? P::neg(ca) : ca;
        }
        if (mdb != INT_MIN) {
          const uint32_t at = base + __popc(ba) + __popc(bb & below);
          lr[at] = tb + (mdb >> 1);
          lc[at] = (mdb & 1) ? P::neg(cb) : cb;
        }
        if (lane == 0) ln[q] = (int)(nh + __popc(ba) + __popc(bb));
      }
    }
    uint32_t nm = 0;
    if (F.mx_ptr) {
      const uint32_t m0 = F.mx_ptr[u];
      nm = F.mx_ptr[u + 1] - m0;
      for (uint32_t k = threadIdx.x; k < nm; k += BS) {
        mr[k] = (uint64_t)F.mx_tgt[m0 + k] * D;
        mc[k] = P::ld(F.mx_val, F.mx_val_df, m0 + k);
        mm[k] = mixd ? (uint32_t)F.mx_mv[m0 + k] * (uint32_t)F.np : (uint32_t)F.mx_mv[m0 + k] * D;
      }
    }
    if (threadIdx.x == 0) {
      n_up_s = (int)nh;
      n_mx_s = (int)nm;
      pat_s = F.row_pat[u];
    }
    cp_async_wait_all();
    __syncthreads();

    const C eu = P::ld(F.e_up, F.e_up_df, u);
    const int nup = n_up_s, nmx = n_mx_s;
    const C* ddr = P::ld_ptr(F.dd, F.dd_df) + (uint64_t)pat_s * NE;
    V* yr = y + (uint64_t)u * D;
    for (uint32_t w = warp; w < F.n_win; w += NWARP) {
      const uint32_t ent = w * 32 + lane;   // this lane's four entries
      const uint4 dq = __ldg(F.perm4 + ent);
      // padding entries read at the window's first string (lane 0, slot 0,
      // always a real one), so every term of the window's list stays in bounds
      const uint32_t d0 = __shfl_sync(0xffffffffu, dq.x, 0);
      uint32_t dv[4];
      bool ok[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t d = sel4(dq, e);
        ok[e] = d < D;
        dv[e] = ok[e] ? d : d0;
      }
      C dg[4];
      ld4<C>(ddr + 4 * (uint64_t)ent, dg);
      const uchar4 c4 = __ldg(F.cnt4 + w);
      A acc[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const V xv = xs[dv[e]];
        acc[e] = P::zero();
        P::mac(acc[e], dg[e], xv);
        P::mac(acc[e], eu, xv);
      }
      // down hops: slot counts descend (c0 >= c1 >= c2 >= c3), so the first c3
      // steps serve all four slots, the next c2 - c3 three, and so on
      {
        const uint4* hp = F.hop4 + (uint64_t)w * F.max_cnt * 32 + lane;
        const int c0 = c4.x, c1 = c4.y, c2 = c4.z, c3 = c4.w;
        int k = 0;
#define ED_HOP(E, WD)                                                                     \
  P::mac(acc[E], *reinterpret_cast<const C*>(reinterpret_cast<const unsigned char*>(cs) + ((WD) & 0x1fffu)), \
         *reinterpret_cast<const V*>(reinterpret_cast<const unsigned char*>(xs) + ((WD) >> 13)))
        for (; k < c3; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x); ED_HOP(1, h.y); ED_HOP(2, h.z); ED_HOP(3, h.w);
        }
        for (; k < c2; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x); ED_HOP(1, h.y); ED_HOP(2, h.z);
        }
        for (; k < c1; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x); ED_HOP(1, h.y);
        }
        for (; k < c0; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x);
        }
#undef ED_HOP
      }
      // the row's term list, two terms at a time: up hops and, in a window
      // whose strings share one impurity pattern, that pattern's spin-flip /
      // pair-hop terms
      const uint32_t wp = mixd ? F.wpat[w] : 0xffffffffu;
      const bool uni = wp != 0xffffffffu;
      {
        const int nlw = uni ? ln[wp] : nup;
        const int64_t* lrw = lr + (uni ? wp * lcap : 0u);
        const C* lcw = lc + (uni ? wp * lcap : 0u);
        int k = 0;
        for (; k + 1 < nlw; k += 2) {
          const V* x0 = x + lrw[k];
          const V* x1 = x + lrw[k + 1];
          V a0[4], a1[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            a0[e] = __ldg(x0 + dv[e]);
            a1[e] = __ldg(x1 + dv[e]);
          }
          const C c0 = lcw[k], c1 = lcw[k + 1];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            P::mac(acc[e], c0, a0[e]);
            P::mac(acc[e], c1, a1[e]);
          }
        }
        if (k < nlw) {
          const V* x0 = x + lrw[k];
          const C c0 = lcw[k];
#pragma unroll
          for (int e = 0; e < 4; ++e) P::mac(acc[e], c0, __ldg(x0 + dv[e]));
        }
      }
      // spin-flip / pair-hop in the other windows
      if (nmx && !uni) {
        if (mixd) {
          const uint32_t pd4 = __ldg(F.dpat4 + ent);
          for (int j = 0; j < nmx; ++j) {
            const V* xm = x + mr[j];
            const C cj = mc[j];
            int32_t md[4];
            V xv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              md[e] = ok[e] ? mds[mm[j] + ((pd4 >> (8 * e)) & 255u)] : INT_MIN;
              if (md[e] != INT_MIN) xv[e] = __ldg(xm + (int64_t)dv[e] + (md[e] >> 1));
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (md[e] != INT_MIN) P::mac(acc[e], (md[e] & 1) ? P::neg(cj) : cj, xv[e]);
          }
        } else {
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
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (ok[e]) {
          const V yv = P::out(acc[e]);
          st_stream(yr + dv[e], yv);
          if (F.dotp) P::dot(dacc, xs[dv[e]], yv);
        }
    }
  }
  if (F.dotp) {
    __shared__ A red[BS / 32];
    dacc = P::warp_sum(dacc);
    if (lane == 0) red[warp] = dacc;
    __syncthreads();
    if (warp == 0) {
      A v = lane < NWARP ? red[lane] : P::zero();
      v = P::warp_sum(v);
      if (lane == 0) F.dotp[blockIdx.x] = P::to_double(v);
    }
  }
}

// ---------------------------------------------------------------- two rows
// Two up strings per block: rows A and B share every down hop (same hop word,
// same coefficient, same staged offset), so the two rows are staged
// interleaved ({A, B} per rank for floats, {A.hi, B.hi, A.lo, B.lo} for
// double-float), the coefficients are kept as {hi, hi, lo, lo}, and both rows'
// double-float accumulators advance together (f32x2 instructions for float
// rows, scalar ones for double-float rows).  Hop words, window permutation and
// coefficient loads are shared by the two rows.  It is the default for float
// vectors with double-float sums; for double-float rows (16 bytes per rank)
// two blocks leave the SM little L1 and the single-row kernel is usually
// faster, which the autotuner measures per sector.
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g));
}

template <class P>
struct PairTraits;

template <>
struct PairTraits<PolDF> {
  using PV = float4;  // {A.hi, B.hi, A.lo, B.lo}
  static constexpr bool XLO = true;
  __device__ static __forceinline__ float2 hi(const PV& v) { return make_float2(v.x, v.y); }
  __device__ static __forceinline__ float2 lo(const PV& v) { return make_float2(v.z, v.w); }
  __device__ static __forceinline__ float2 hi2(float2 a, float2 b) { return make_float2(a.x, b.x); }
  __device__ static __forceinline__ float2 lo2(float2 a, float2 b) { return make_float2(a.y, b.y); }
  __device__ static __forceinline__ void stage(PV* s, const float2* a, const float2* b) {
    cp_async4(&s->x, &a->x);
    cp_async4(&s->y, &b->x);
    cp_async4(&s->z, &a->y);
    cp_async4(&s->w, &b->y);
  }
  __device__ static __forceinline__ float2 out(float h, float l) { return df_norm(make_float2(h, l)); }
  __device__ static __forceinline__ float2 xa(const PV& v) { return make_float2(v.x, v.z); }
  __device__ static __forceinline__ float2 xb(const PV& v) { return make_float2(v.y, v.w); }
};

template <>
struct PairTraits<PolF32> {
  using PV = float2;  // {A, B}
  static constexpr bool XLO = false;
  __device__ static __forceinline__ float2 hi(const PV& v) { return v; }
  __device__ static __forceinline__ float2 lo(const PV&) { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ float2 hi2(float a, float b) { return make_float2(a, b); }
  __device__ static __forceinline__ float2 lo2(float, float) { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ void stage(PV* s, const float* a, const float* b) {
    cp_async4(&s->x, a);
    cp_async4(&s->y, b);
  }
  __device__ static __forceinline__ float out(float h, float l) { return __fadd_rn(h, l); }
  __device__ static __forceinline__ float xa(const PV& v) { return v.x; }
  __device__ static __forceinline__ float xb(const PV& v) { return v.y; }
};

template <class P>
size_t pair_smem(uint32_t D, int n_coef) {
  return align16(D * sizeof(typename PairTraits<P>::PV)) + align16((size_t)n_coef * 16) + 4 * align16(kList * 16) +
         align16(kList * 8) + align16(kMaxDelta * 4);
}

// The two rows' multiply-adds of a pair, lane-wise exactly df_mac (XLO, x in
// double-float) or df_mac1 (float x).  Double-float rows run them as scalar
// FP32 instructions (0.70 ms against 0.78 ms with f32x2 at N_s = 15), float
// rows as f32x2 instructions (0.49 ms against 0.55 ms scalar).
template <bool XLO>
__device__ __forceinline__ void df_mac2s(float2& H, float2& L, float2 Ch, float2 Cl, float2 Xh, float2 Xl) {
  if (XLO) {
    float2 a = make_float2(H.x, L.x), b = make_float2(H.y, L.y);
    df_mac(a, make_float2(Ch.x, Cl.x), make_float2(Xh.x, Xl.x));
    df_mac(b, make_float2(Ch.y, Cl.y), make_float2(Xh.y, Xl.y));
    H = make_float2(a.x, b.x);
    L = make_float2(a.y, b.y);
  } else {
    df_mac2<false>(H, L, Ch, Cl, Xh, Xl);
  }
}

// coefficient pair (sa * c_A, sb * c_B) from a {A.hi, B.hi, A.lo, B.lo} entry, sa, sb in {0, 1, -1}
__device__ __forceinline__ float4 sign_pair(float4 c, int32_t mda, int32_t mdb) {
  if (mda == INT_MIN) c.x = c.z = 0.f;
  else if (mda & 1) c.x = -c.x, c.z = -c.z;
  if (mdb == INT_MIN) c.y = c.w = 0.f;
  else if (mdb & 1) c.y = -c.y, c.w = -c.w;
  return c;
}

template <class P, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_apply_pair(FastView F, const typename P::V* __restrict__ x,
                                                        typename P::V* __restrict__ y) {
  using V = typename P::V;
  using A = typename P::A;
  using T = PairTraits<P>;
  using PV = typename T::PV;
  constexpr bool XLO = T::XLO;
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t D = F.D;
  unsigned char* p = sm;
  PV* xs = reinterpret_cast<PV*>(p);            // interleaved rows A and B
  p += align16(D * sizeof(PV));
  float4* cs = reinterpret_cast<float4*>(p);    // {hi, hi, lo, lo} per distinct down-hop element
  p += align16((size_t)F.n_coef * 16);
  float4* lc = reinterpret_cast<float4*>(p);    // up-hop coefficients {A.hi, B.hi, A.lo, B.lo}
  p += align16(kList * 16);
  float4* mc = reinterpret_cast<float4*>(p);    // mixed coefficients, same layout
  p += align16(kList * 16);
  ulonglong2* lr = reinterpret_cast<ulonglong2*>(p);  // up-hop row offsets (elements) of A and B
  p += align16(kList * 16);
  ulonglong2* mr = reinterpret_cast<ulonglong2*>(p);  // mixed row offsets
  p += align16(kList * 16);
  uint2* mm = reinterpret_cast<uint2*>(p);            // mixed move offsets, ~0u for padding
  p += align16(kList * 8);
  int32_t* mds = reinterpret_cast<int32_t*>(p);       // move shifts per pattern
  __shared__ int n_up_s, n_mx_s;
  __shared__ uint32_t pat_s[2];
  const bool mixd = F.dpat4 != nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NWARP = BS / 32;
  const uint64_t NE = (uint64_t)F.n_win * kWin;
  constexpr uint32_t kPad = 0xffffffffu;

  for (int k = threadIdx.x; k < F.n_coef; k += BS) {
    const float2 c = F.coef_df[k];
    cs[k] = make_float4(c.x, c.x, c.y, c.y);
  }
  for (int k = threadIdx.x; k < F.n_md; k += BS) mds[k] = F.mdelta[k];
  A dacc = P::zero();  // <x, y> over this thread's elements (only used with F.dotp)

  const uint32_t n_pairs = (F.D_up + 1) / 2;
  for (uint32_t i = blockIdx.x; i < n_pairs; i += gridDim.x) {
    const uint32_t uA = F.row_order[2 * i];
    const bool hasB = 2 * i + 1 < F.D_up;
    const uint32_t uB = hasB ? F.row_order[2 * i + 1] : uA;
    __syncthreads();
    {
      const V* xa = x + (uint64_t)uA * D;
      const V* xb = x + (uint64_t)uB * D;
      for (uint32_t d = threadIdx.x; d < D; d += BS) T::stage(xs + d, xa + d, xb + d);
    }
    // up-hop lists of A and B side by side; the shorter one is padded with a
    // zero coefficient on its own row
    const uint32_t a0 = F.uh_ptr[uA], na = F.uh_ptr[uA + 1] - a0;
    const uint32_t b0 = F.uh_ptr[uB], nb = hasB ? F.uh_ptr[uB + 1] - b0 : 0u;
    const uint32_t nh = na > nb ? na : nb;
    for (uint32_t k = threadIdx.x; k < nh; k += BS) {
      const float2 ca = k < na ? F.uh_val_df[a0 + k] : make_float2(0.f, 0.f);
      const float2 cb = k < nb ? F.uh_val_df[b0 + k] : make_float2(0.f, 0.f);
      lr[k] = make_ulonglong2((unsigned long long)(k < na ? F.uh_tgt[a0 + k] : uA) * D,
                              (unsigned long long)(k < nb ? F.uh_tgt[b0 + k] : uB) * D);
      lc[k] = make_float4(ca.x, cb.x, ca.y, cb.y);
    }
    uint32_t nm = 0;
    if (F.mx_ptr) {
      const uint32_t ma0 = F.mx_ptr[uA], ma = F.mx_ptr[uA + 1] - ma0;
      const uint32_t mb0 = F.mx_ptr[uB], mb = hasB ? F.mx_ptr[uB + 1] - mb0 : 0u;
      nm = ma > mb ? ma : mb;
      const uint32_t stride = mixd ? (uint32_t)F.np : D;
      for (uint32_t k = threadIdx.x; k < nm; k += BS) {
        const float2 ca = k < ma ? F.mx_val_df[ma0 + k] : make_float2(0.f, 0.f);
        const float2 cb = k < mb ? F.mx_val_df[mb0 + k] : make_float2(0.f, 0.f);
        mr[k] = make_ulonglong2((unsigned long long)(k < ma ? F.mx_tgt[ma0 + k] : uA) * D,
                                (unsigned long long)(k < mb ? F.mx_tgt[mb0 + k] : uB) * D);
        mc[k] = make_float4(ca.x, cb.x, ca.y, cb.y);
        mm[k] = make_uint2(k < ma ? (uint32_t)F.mx_mv[ma0 + k] * stride : kPad,
                           k < mb ? (uint32_t)F.mx_mv[mb0 + k] * stride : kPad);
      }
    }
    if (threadIdx.x == 0) {
      n_up_s = (int)nh;
      n_mx_s = (int)nm;
      pat_s[0] = F.row_pat[uA];
      pat_s[1] = F.row_pat[uB];
    }
    cp_async_wait_all();
    __syncthreads();

    const float2 euA = F.e_up_df[uA], euB = F.e_up_df[uB];
    const float2 EUh = make_float2(euA.x, euB.x), EUl = make_float2(euA.y, euB.y);
    const int nup = n_up_s, nmx = n_mx_s;
    const float2* ddA = F.dd_df + (uint64_t)pat_s[0] * NE;
    const float2* ddB = F.dd_df + (uint64_t)pat_s[1] * NE;
    V* yA = y + (uint64_t)uA * D;
    V* yB = y + (uint64_t)uB * D;
    for (uint32_t w = warp; w < F.n_win; w += NWARP) {
      const uint32_t ent = w * 32 + lane;  // this lane's four entries
      const uint4 dq = __ldg(F.perm4 + ent);
      uint32_t dv[4];
      bool ok[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t d = sel4(dq, e);
        ok[e] = d < D;
        dv[e] = ok[e] ? d : 0u;
      }
      float2 dga[4], dgb[4];
      ld4<float2>(ddA + 4 * (uint64_t)ent, dga);
      ld4<float2>(ddB + 4 * (uint64_t)ent, dgb);
      float2 H[4], L[4];  // (A, B) hi and lo parts of the four slots
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const PV X = xs[dv[e]];
        H[e] = L[e] = make_float2(0.f, 0.f);
        df_mac2s<XLO>(H[e], L[e], make_float2(dga[e].x, dgb[e].x), make_float2(dga[e].y, dgb[e].y), T::hi(X),
                     T::lo(X));
        df_mac2s<XLO>(H[e], L[e], EUh, EUl, T::hi(X), T::lo(X));
      }
      // down hops: slot counts descend (c0 >= c1 >= c2 >= c3)
      {
        const uchar4 c4 = __ldg(F.cnt4 + w);
        const uint4* hp = F.hop4 + (uint64_t)w * F.max_cnt * 32 + lane;
        const int c0 = c4.x, c1 = c4.y, c2 = c4.z, c3 = c4.w;
        int k = 0;
#define ED_HOP(E, WD)                                                                                      \
  do {                                                                                                     \
    const float4 cc = *reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(cs) + ((WD) & 0x1fffu)); \
    const PV X = *reinterpret_cast<const PV*>(reinterpret_cast<const unsigned char*>(xs) + ((WD) >> 13));  \
    df_mac2s<XLO>(H[E], L[E], make_float2(cc.x, cc.y), make_float2(cc.z, cc.w), T::hi(X), T::lo(X));        \
  } while (0)
        for (; k < c3; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x); ED_HOP(1, h.y); ED_HOP(2, h.z); ED_HOP(3, h.w);
        }
        for (; k < c2; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x); ED_HOP(1, h.y); ED_HOP(2, h.z);
        }
        for (; k < c1; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x); ED_HOP(1, h.y);
        }
        for (; k < c0; ++k) {
          const uint4 h = __ldg(hp + (uint64_t)k * 32);
          ED_HOP(0, h.x);
        }
#undef ED_HOP
      }
      // up hops: the k-th neighbour row of A and of B
      for (int k = 0; k < nup; ++k) {
        const ulonglong2 R = lr[k];
        const float4 cc = lc[k];
        V a[4], b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a[e] = __ldg(x + R.x + dv[e]);
          b[e] = __ldg(x + R.y + dv[e]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
          df_mac2s<XLO>(H[e], L[e], make_float2(cc.x, cc.y), make_float2(cc.z, cc.w), T::hi2(a[e], b[e]),
                       T::lo2(a[e], b[e]));
      }
      // spin-flip / pair-hop
      if (nmx) {
        const uint32_t wp = mixd ? F.wpat[w] : 0xffffffffu;
        if (wp != 0xffffffffu) {
          // every string of the window has impurity pattern wp: one shift per row
          for (int j = 0; j < nmx; ++j) {
            const uint2 M = mm[j];
            const int32_t mda = M.x != kPad ? mds[M.x + wp] : INT_MIN;
            const int32_t mdb = M.y != kPad ? mds[M.y + wp] : INT_MIN;
            if (mda == INT_MIN && mdb == INT_MIN) continue;
            const ulonglong2 R = mr[j];
            const float4 cc = sign_pair(mc[j], mda, mdb);
            const V* xa = x + R.x + (mda == INT_MIN ? 0 : (mda >> 1));
            const V* xb = x + R.y + (mdb == INT_MIN ? 0 : (mdb >> 1));
            V a[4], b[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              a[e] = ok[e] ? __ldg(xa + dv[e]) : x[0];
              b[e] = ok[e] ? __ldg(xb + dv[e]) : x[0];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
              df_mac2s<XLO>(H[e], L[e], make_float2(cc.x, cc.y), make_float2(cc.z, cc.w), T::hi2(a[e], b[e]),
                           T::lo2(a[e], b[e]));
          }
        } else {
          // per-lane shifts: from the entry's impurity pattern, or the generic move tables
          const uint32_t pd4 = mixd ? __ldg(F.dpat4 + ent) : 0u;
          for (int j = 0; j < nmx; ++j) {
            const uint2 M = mm[j];
            const ulonglong2 R = mr[j];
            const float4 c0 = mc[j];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              int32_t mda = INT_MIN, mdb = INT_MIN;
              uint64_t ia = 0, ib = 0;
              if (ok[e]) {
                if (mixd) {
                  const uint32_t pe = (pd4 >> (8 * e)) & 255u;
                  if (M.x != kPad) mda = mds[M.x + pe];
                  if (M.y != kPad) mdb = mds[M.y + pe];
                  if (mda != INT_MIN) ia = R.x + (uint64_t)((int64_t)dv[e] + (mda >> 1));
                  if (mdb != INT_MIN) ib = R.y + (uint64_t)((int64_t)dv[e] + (mdb >> 1));
                } else {
                  if (M.x != kPad) {
                    const int32_t v = __ldg(F.mv + M.x + dv[e]);
                    if (v >= 0) mda = v, ia = R.x + (uint32_t)(v >> 1);
                  }
                  if (M.y != kPad) {
                    const int32_t v = __ldg(F.mv + M.y + dv[e]);
                    if (v >= 0) mdb = v, ib = R.y + (uint32_t)(v >> 1);
                  }
                }
              }
              if (mda == INT_MIN && mdb == INT_MIN) continue;
              const float4 cc = sign_pair(c0, mda, mdb);
              const V a = __ldg(x + ia), b = __ldg(x + ib);
              df_mac2s<XLO>(H[e], L[e], make_float2(cc.x, cc.y), make_float2(cc.z, cc.w), T::hi2(a, b),
                           T::lo2(a, b));
            }
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (ok[e]) {
          const V ya = T::out(H[e].x, L[e].x);
          st_stream(yA + dv[e], ya);
          if (F.dotp) P::dot(dacc, T::xa(xs[dv[e]]), ya);
          if (hasB) {
            const V yb = T::out(H[e].y, L[e].y);
            st_stream(yB + dv[e], yb);
            if (F.dotp) P::dot(dacc, T::xb(xs[dv[e]]), yb);
          }
        }
    }
  }
  if (F.dotp) {
    __shared__ A red[BS / 32];
    dacc = P::warp_sum(dacc);
    if (lane == 0) red[warp] = dacc;
    __syncthreads();
    if (warp == 0) {
      A v = lane < NWARP ? red[lane] : P::zero();
      v = P::warp_sum(v);
      if (lane == 0) F.dotp[blockIdx.x] = P::to_double(v);
    }
  }
}

// Window tables: entry idx = w*128 + lane*4 + slot holds down rank perm[idx]
// (D for padding).  Hop words of entry idx at [w][k][lane][slot].
__global__ void k_win_tables(uint32_t D, uint32_t n_win, uint32_t max_cnt, const uint32_t* __restrict__ perm,
                             const uint32_t* __restrict__ dbasis, const uint32_t* __restrict__ dh_ptr,
                             const uint32_t* __restrict__ dh_tgt, const double* __restrict__ dh_val,
                             const double* __restrict__ coef, int n_coef, int zero_id, int vbytes, int cbytes,
                             uint32_t* __restrict__ hop, const double* __restrict__ e_dn,
                             const double* __restrict__ W, int w_lo, int wbits, int n_pat, double* __restrict__ dd,
                             int orb0, uint8_t* __restrict__ dpat) {
  const uint64_t NE = (uint64_t)n_win * kWin;
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NE) return;
  const uint32_t w = (uint32_t)(idx / kWin), r = (uint32_t)(idx % kWin);  // r = lane*4 + slot
  const uint32_t d = perm[idx];
  const bool real = d < D;
  const uint32_t h0 = real ? dh_ptr[d] : 0u, c = real ? dh_ptr[d + 1] - h0 : 0u;
  for (uint32_t k = 0; k < max_cnt; ++k) {
    // shared-memory byte offsets: x element << 13 | coefficient
    uint32_t word = (uint32_t)(zero_id * cbytes);  // element 0 times the zero coefficient
    if (k < c) {
      const double v = dh_val[h0 + k];
      int id = 0;
      while (id < n_coef && coef[id] != v) ++id;
      word = ((dh_tgt[h0 + k] * (uint32_t)vbytes) << 13) | (uint32_t)(id * cbytes);
    }
    hop[((uint64_t)w * max_cnt + k) * kWin + r] = word;
  }
  const uint32_t s = real ? dbasis[d] : 0u;
  const uint32_t pd = (wbits > 0) ? ((s >> w_lo) & ((1u << wbits) - 1u)) : 0u;
  for (int pu = 0; pu < n_pat; ++pu) {
    double v = 0.0;
    if (real) {
      v = e_dn[d];
      if (W) v += W[((uint32_t)pu << wbits) + pd];
    }
    dd[(uint64_t)pu * NE + idx] = v;
  }
  if (dpat) dpat[idx] = (uint8_t)(real ? (s >> orb0) : 0u);
}

// Rank shift of each impurity move (x -> y) for each pattern p, read off the
// move table at one string of pattern p (the shift is the same for every
// string of the pattern when the orbitals are the top sites); INT_MIN where
// the move does not apply.
__global__ void k_mix_delta(uint32_t D, const uint32_t* __restrict__ dbasis, const int32_t* __restrict__ mv,
                            int orb0, int M, int32_t* __restrict__ mdelta) {
  const int NP = 1 << M;
  for (int idx = threadIdx.x; idx < M * M * NP; idx += blockDim.x) {
    const int move = idx / NP, p = idx % NP;
    int32_t out = INT_MIN;
    for (uint32_t d = 0; d < D; ++d) {
      if ((int)(dbasis[d] >> orb0) != p) continue;
      const int32_t v = mv[(uint64_t)move * D + d];
      if (v >= 0) out = (int32_t)(((int64_t)(v >> 1) - (int64_t)d) * 2 + (v & 1));
      break;
    }
    mdelta[idx] = out;
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
  F.n_win = f.n_win;
  F.max_cnt = f.max_cnt;
  F.row_order = f.row_order;
  F.row_pat = f.row_pat;
  F.perm4 = reinterpret_cast<const uint4*>(f.perm);
  F.cnt4 = reinterpret_cast<const uchar4*>(f.cnt);
  F.hop4 = reinterpret_cast<const uint4*>(f.hop);
  F.coef = f.coef;
  F.coef_df = f.coef_df;
  F.n_coef = f.n_coef;
  F.dd = f.dd;
  F.dd_df = f.dd_df;
  F.mv = s->dn_move;
  F.dpat4 = f.mix_delta ? reinterpret_cast<const uint32_t*>(f.dpat) : nullptr;
  F.wpat = f.mix_delta ? f.wpat : nullptr;
  F.mdelta = f.mix_delta ? f.mdelta : nullptr;
  F.np = 1 << s->M;
  F.n_md = f.mix_delta ? s->M * s->M * (1 << s->M) : 0;
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
  F.n_lp = f.n_lp;
  F.lcap = f.lcap;
  return F;
}

template <class P, int BS, int MINB>
int launch_fast(const Sector* s, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts) {
  FastView F = make_view<P>(s);
  F.dotp = dotp;
  size_t smem = fast_smem<P>(F.D, F.n_coef, F.n_lp, F.lcap);
  auto kern = k_apply_win<P, BS, MINB>;
  ED_TRY(smem_cap(s->ctx, kern, smem));
  int per_sm = 0;
  ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem));
  if (per_sm < 1) ED_INVALID("fast row kernel does not fit on an SM (%zu B shared)", smem);
  uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)s->ctx->num_sms * per_sm, F.D_up);
  kern<<<grid, BS, smem, st>>>(F, static_cast<const typename P::V*>(x), static_cast<typename P::V*>(y));
  ED_LAUNCH_CHECK();
  if (nparts) *nparts = (int)grid;
  return ED_OK;
}

template <class P, int BS, int MINB>
int launch_pair(const Sector* s, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts) {
  if (!s->fast.pair_ok) ED_INVALID("the sector has no two-row kernel tables");
  FastView F = make_view<P>(s);
  F.hop4 = reinterpret_cast<const uint4*>(s->fast.hop2);
  F.dotp = dotp;
  size_t smem = pair_smem<P>(F.D, F.n_coef);
  auto kern = k_apply_pair<P, BS, MINB>;
  ED_TRY(smem_cap(s->ctx, kern, smem));
  int per_sm = 0;
  ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem));
  if (per_sm < 1) ED_INVALID("two-row kernel does not fit on an SM (%zu B shared)", smem);
  uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)s->ctx->num_sms * per_sm, (F.D_up + 1) / 2);
  kern<<<grid, BS, smem, st>>>(F, static_cast<const typename P::V*>(x), static_cast<typename P::V*>(y));
  ED_LAUNCH_CHECK();
  if (nparts) *nparts = (int)grid;
  return ED_OK;
}

// H*v variants of the fast path: up strings per block (one: k_apply_win, two:
// k_apply_pair) times a launch shape (threads per block, the blocks per SM the
// register budget is sized for; shared memory may allow fewer).
constexpr int kNShapes = 5;
constexpr int kShapeBS[kNShapes] = {256, 192, 256, 512, 384};
constexpr int kShapeMinB[kNShapes] = {3, 4, 2, 1, 2};

template <class P>
int run_variant(const Sector* s, int v, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts) {
  switch (v) {
    case 0: return launch_fast<P, 256, 3>(s, x, y, st, dotp, nparts);
    case 1: return launch_fast<P, 192, 4>(s, x, y, st, dotp, nparts);
    case 2: return launch_fast<P, 256, 2>(s, x, y, st, dotp, nparts);
    case 3: return launch_fast<P, 512, 1>(s, x, y, st, dotp, nparts);
    case 4: return launch_fast<P, 384, 2>(s, x, y, st, dotp, nparts);
  }
  if constexpr (P::prec != ED_PREC_FP64) {
    switch (v) {
      case 5: return launch_pair<P, 256, 3>(s, x, y, st, dotp, nparts);
      case 6: return launch_pair<P, 192, 4>(s, x, y, st, dotp, nparts);
      case 7: return launch_pair<P, 256, 2>(s, x, y, st, dotp, nparts);
      case 8: return launch_pair<P, 512, 1>(s, x, y, st, dotp, nparts);
      case 9: return launch_pair<P, 384, 2>(s, x, y, st, dotp, nparts);
    }
  }
  ED_INVALID("H*v variant %d does not apply to this sector", v);
}

}  // namespace

int build_fast(Sector* s) {
  s->fast.ok = false;
  const uint32_t D = s->dn.D;
  if (D < 512 || s->n_chunks > 1 || s->up.max_hops > (uint32_t)kList || s->max_mix > (uint32_t)kList)
    return ED_OK;
  if (s->dn.max_hops > 255) return ED_OK;
  if (s->dn_move && s->M * s->M > kList) return ED_OK;
  // distinct down-hop matrix elements plus a zero used for padding
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
  int zero_id = -1;
  for (size_t i = 0; i < coef.size(); ++i)
    if (coef[i] == 0.0) zero_id = (int)i;
  if (zero_id < 0) {
    if (coef.size() >= (size_t)kMaxCoef) return ED_OK;
    zero_id = (int)coef.size();
    coef.push_back(0.0);
  }
  // single-row tables always; two-row tables (double-float and float rows)
  // where two interleaved rows fit.  Hop words address the staged row in
  // bytes below 2^19.
  const size_t vbytes = elem_bytes(s->prec);
  if ((uint64_t)D * vbytes >= (1ull << 19)) return ED_OK;
  const int nc = (int)coef.size();
  const bool mix_delta = s->dn_move && s->orb0 + s->M == s->n_s && s->M * s->M * (1 << s->M) <= kMaxDelta;
  const int n_lp = mix_delta ? 1 << s->M : 1;
  const uint32_t lcap = std::max(1u, s->up.max_hops + (mix_delta ? s->max_mix : 0u));
  if (std::max(fast_smem<PolF64>(D, nc, n_lp, lcap), fast_smem<PolDF>(D, nc, n_lp, lcap)) > 220 * 1024) return ED_OK;
  const size_t smem2 = s->prec == ED_PREC_DF64 ? pair_smem<PolDF>(D, nc) : pair_smem<PolF32>(D, nc);
  const bool pair = s->prec != ED_PREC_FP64 && (uint64_t)D * 2 * vbytes < (1ull << 19) && smem2 <= 220 * 1024;

  // window-local order: inside each window of 128 ranks, longest hop list first
  const uint32_t n_win = (D + kWin - 1) / kWin;
  std::vector<uint32_t> dptr(D + 1);
  ED_TRY_CUDA(cudaMemcpy(dptr.data(), s->dn.hop_ptr, sizeof(uint32_t) * (D + 1), cudaMemcpyDeviceToHost));
  std::vector<uint32_t> perm((size_t)n_win * kWin, D);
  std::vector<uint8_t> cnt((size_t)n_win * 4, 0);
  for (uint32_t w = 0; w < n_win; ++w) {
    std::vector<uint32_t> ds;
    for (uint32_t d = w * kWin; d < std::min(D, (w + 1) * kWin); ++d) ds.push_back(d);
    std::stable_sort(ds.begin(), ds.end(), [&](uint32_t a, uint32_t b) {
      return (dptr[a + 1] - dptr[a]) > (dptr[b + 1] - dptr[b]);
    });
    for (size_t r = 0; r < ds.size(); ++r) {
      const uint32_t slot = (uint32_t)(r / 32), lane = (uint32_t)(r % 32);
      perm[(size_t)w * kWin + lane * 4 + slot] = ds[r];
      uint8_t& c = cnt[(size_t)w * 4 + slot];
      c = (uint8_t)std::max<uint32_t>(c, dptr[ds[r] + 1] - dptr[ds[r]]);
    }
  }

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
  {
    // inside a component, rows with equal up-hop and mixed-list lengths sit
    // next to each other, so the two rows of a pair pad their lists little
    std::vector<uint32_t> uptr(Du + 1), mptr;
    ED_TRY_CUDA(cudaMemcpy(uptr.data(), s->up.hop_ptr, sizeof(uint32_t) * (Du + 1), cudaMemcpyDeviceToHost));
    if (s->mx_ptr) {
      mptr.resize(Du + 1);
      ED_TRY_CUDA(cudaMemcpy(mptr.data(), s->mx_ptr, sizeof(uint32_t) * (Du + 1), cudaMemcpyDeviceToHost));
    }
    auto lens = [&](uint32_t u) {
      return std::make_pair(uptr[u + 1] - uptr[u], mptr.empty() ? 0u : mptr[u + 1] - mptr[u]);
    };
    std::stable_sort(rorder.begin(), rorder.end(), [&](uint32_t a, uint32_t b) {
      if (rkey[a] != rkey[b]) return rkey[a] < rkey[b];
      return lens(a) < lens(b);
    });
  }

  auto& f = s->fast;
  const int wbits = (s->n_chunks == 1) ? s->w_bits[0] : 0;
  f.n_win = n_win;
  f.max_cnt = std::max(1u, s->dn.max_hops);
  f.n_coef = (int)coef.size();
  f.n_pat = 1 << wbits;
  f.n_lp = n_lp;
  f.lcap = lcap;
  const uint64_t NE = (uint64_t)n_win * kWin;
  ED_TRY(sector_alloc(s, &f.perm, NE));
  ED_TRY(sector_alloc(s, &f.cnt, (size_t)n_win * 4));
  ED_TRY(sector_alloc(s, &f.hop, (size_t)f.max_cnt * NE));
  ED_TRY(sector_alloc(s, &f.coef, f.n_coef));
  ED_TRY(sector_alloc(s, &f.dd, (size_t)f.n_pat * NE));
  ED_TRY(sector_alloc(s, &f.row_order, Du));
  ED_TRY(sector_alloc(s, &f.row_pat, Du));
  ED_TRY_CUDA(cudaMemcpy(f.perm, perm.data(), sizeof(uint32_t) * NE, cudaMemcpyHostToDevice));
  ED_TRY_CUDA(cudaMemcpy(f.cnt, cnt.data(), cnt.size(), cudaMemcpyHostToDevice));
  ED_TRY_CUDA(cudaMemcpy(f.coef, coef.data(), sizeof(double) * f.n_coef, cudaMemcpyHostToDevice));
  ED_TRY_CUDA(cudaMemcpy(f.row_order, rorder.data(), sizeof(uint32_t) * Du, cudaMemcpyHostToDevice));
  f.mix_delta = mix_delta;
  f.pair_ok = pair;
  if (mix_delta) {
    const int M = s->M, NP = 1 << M;
    std::vector<uint32_t> dbas(D), wpat(n_win, 0xffffffffu);
    ED_TRY_CUDA(cudaMemcpy(dbas.data(), s->dn.basis, sizeof(uint32_t) * D, cudaMemcpyDeviceToHost));
    for (uint32_t w = 0; w < n_win; ++w) {
      uint32_t p0 = dbas[w * kWin] >> s->orb0;
      bool same = true;
      for (uint32_t d = w * kWin; d < std::min(D, (w + 1) * kWin); ++d) same = same && ((dbas[d] >> s->orb0) == p0);
      if (same) wpat[w] = p0;
    }
    ED_TRY(sector_alloc(s, &f.wpat, n_win));
    ED_TRY_CUDA(cudaMemcpy(f.wpat, wpat.data(), sizeof(uint32_t) * n_win, cudaMemcpyHostToDevice));
    ED_TRY(sector_alloc(s, &f.dpat, NE));
    ED_TRY(sector_alloc(s, &f.mdelta, (size_t)M * M * NP));
    k_mix_delta<<<1, 256>>>(D, s->dn.basis, s->dn_move, s->orb0, M, f.mdelta);
    ED_LAUNCH_CHECK();
  }
  k_win_tables<<<(unsigned)((NE + 127) / 128), 128>>>(D, n_win, f.max_cnt, f.perm, s->dn.basis, s->dn.hop_ptr,
                                                      s->dn.hop_tgt, s->dn.hop_val, f.coef, f.n_coef, zero_id,
                                                      (int)vbytes, 8,
                                                      f.hop, s->dn.e, (s->n_chunks == 1) ? s->W : nullptr, s->w_lo,
                                                      wbits, f.n_pat, f.dd, s->orb0, f.dpat);
  if (pair) {
    ED_TRY(sector_alloc(s, &f.hop2, (size_t)f.max_cnt * NE));
    k_win_tables<<<(unsigned)((NE + 127) / 128), 128>>>(D, n_win, f.max_cnt, f.perm, s->dn.basis, s->dn.hop_ptr,
                                                        s->dn.hop_tgt, s->dn.hop_val, f.coef, f.n_coef, zero_id,
                                                        (int)(2 * vbytes), 16, f.hop2, s->dn.e, nullptr, s->w_lo,
                                                        wbits, 0, nullptr, s->orb0, nullptr);
  }
  ED_LAUNCH_CHECK();
  k_row_pat<<<(Du + 127) / 128, 128>>>(Du, s->up.basis, s->w_lo, wbits, f.row_pat);
  ED_LAUNCH_CHECK();
  if (s->prec != ED_PREC_FP64) {
    ED_TRY(sector_alloc(s, &f.coef_df, f.n_coef));
    ED_TRY(sector_alloc(s, &f.dd_df, (size_t)f.n_pat * NE));
    k_df_copy<<<(f.n_coef + 127) / 128, 128>>>(f.coef, f.coef_df, f.n_coef);
    k_df_copy<<<(unsigned)(((uint64_t)f.n_pat * NE + 255) / 256), 256>>>(f.dd, f.dd_df, (uint64_t)f.n_pat * NE);
    ED_LAUNCH_CHECK();
  }
  ED_TRY_CUDA(cudaStreamSynchronize(0));  // legacy stream only: leaves other work running
  f.ok = true;
  ED_TRY(build_nat(s, coef, zero_id));
  tune_apply_cached(s);  // a variant tuned earlier for this shape (any creator: ABI, server, Green's function)
  return ED_OK;
}

// Variant index: [0, 5) single-row kernel, [5, 10) two-row kernel (launch
// shapes of kShapeBS / kShapeMinB), [10, 16) natural-order kernel
// (apply_nat.cu).  Float sectors with natural-order tables use only the last
// group, whose float sums differ from the double-float sums of the others;
// double-float sectors may use all three (the natural-order kernel sums in
// another order, within the format's rounding).  Within each group every
// variant gives the same y bit for bit.
constexpr int kNatBase = 2 * kNShapes;

int fast_variants() { return kNatBase + kNatVariants; }

void fast_variant_info(int prec, int v, int* kernel, int* block, int* min_blocks) {
  if (v >= kNatBase) {
    int rows = 0;
    nat_variant_info(prec, v - kNatBase, &rows, block, min_blocks);
    *kernel = 4;
    return;
  }
  *kernel = v < kNShapes ? 2 : 3;
  *block = kShapeBS[v % kNShapes];
  *min_blocks = kShapeMinB[v % kNShapes];
}

bool fast_variant_applies(const Sector* s, int v) {
  if (!s->fast.ok || v < 0 || v >= fast_variants()) return false;
  if (v >= kNatBase)  // the rows a block stages must fit its shared memory
    return s->fast.nat_ok && nat_variant_smem(s, v - kNatBase) + 1024 <= s->ctx->smem_optin;
  // float sectors with natural-order tables keep its float sums whatever the tuning
  if (s->fast.nat_ok && s->prec == ED_PREC_FP32) return false;
  return v < kNShapes || s->fast.pair_ok;
}

// Untuned choice: the natural-order kernel for float sectors that have it
// (four or two rows per block, by what the SM's shared memory holds);
// otherwise two rows per block for float vectors, one otherwise; 256
// threads x 3 blocks per SM while three staged blocks fit the SM's shared
// memory, else 384 x 2 (24 warps either way; measured at N_s = 16, where
// 384 x 2 beats 256 x 2 by ~20%).
int fast_default_variant(const Sector* s) {
  if (s->fast.nat_ok && s->prec == ED_PREC_FP32) {
    // four rows per block and 32 warps per SM: 512 x 2 where two such blocks
    // fit an SM (N_s = 15: 0.279 ms against 0.332 ms for two rows, 256 x 3),
    // else 1024 x 1 where one fits (N_s = 16: 1.31 ms against 1.63 ms for two
    // rows, 512 x 2), as long as the rows give every SM its blocks; else two
    // rows, 256 x 3 where three blocks fit, else 512 x 2
    const size_t per_sm = s->ctx->smem_per_sm ? s->ctx->smem_per_sm : 228 * 1024;
    const uint32_t sms = s->ctx->num_sms > 0 ? (uint32_t)s->ctx->num_sms : 152u;
    const uint32_t tiles4 = (s->up.D + 3) / 4;
    if (2 * (nat_variant_smem(s, 1) + 1024) <= per_sm && tiles4 >= 2 * sms) return kNatBase + 1;
    if (nat_variant_smem(s, 0) + 1024 <= std::min(per_sm, s->ctx->smem_optin) && tiles4 >= sms) return kNatBase + 0;
    return kNatBase + (3 * (nat_variant_smem(s, 3) + 1024) <= per_sm ? 3 : 4);
  }
  const bool pair = s->prec == ED_PREC_FP32 && s->fast.pair_ok;
  const uint32_t D = s->dn.D;
  const int nc = s->fast.n_coef;
  size_t smem = 0;
  if (pair) smem = pair_smem<PolF32>(D, nc);
  else if (s->prec == ED_PREC_FP64) smem = fast_smem<PolF64>(D, nc, s->fast.n_lp, s->fast.lcap);
  else smem = fast_smem<PolDF>(D, nc, s->fast.n_lp, s->fast.lcap);
  const size_t per_sm = s->ctx->smem_per_sm ? s->ctx->smem_per_sm : 228 * 1024;
  const bool three = 3 * (smem + 1024) <= per_sm;  // 1 KB reserved per block
  return (pair ? kNShapes : 0) + (three ? 0 : 4);   // shape 0: 256 x 3, shape 4: 384 x 2
}

int apply_fast_variant(const Sector* s, int v, const void* x, void* y, cudaStream_t st, double* dotp,
                       int* nparts) {
  if (!fast_variant_applies(s, v)) ED_INVALID("H*v variant %d does not apply to this sector", v);
  if (v >= kNatBase) return launch_nat(s, v - kNatBase, x, y, st, dotp, nparts);
  switch (s->prec) {
    case ED_PREC_FP64: return run_variant<PolF64>(s, v, x, y, st, dotp, nparts);
    case ED_PREC_DF64: return run_variant<PolDF>(s, v, x, y, st, dotp, nparts);
    case ED_PREC_FP32: return run_variant<PolF32>(s, v, x, y, st, dotp, nparts);
  }
  ED_INVALID("unknown precision");
}

int apply_fast(const Sector* s, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts) {
  const int v = fast_variant_applies(s, s->tune) ? s->tune : fast_default_variant(s);
  return apply_fast_variant(s, v, x, y, st, dotp, nparts);
}

}  // namespace ed
