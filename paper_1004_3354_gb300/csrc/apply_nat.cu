// H*v in natural order with several up strings per block: the production
// kernel for float (ED_PREC_FP32) and double-float (ED_PREC_DF64) sectors.
//
// The operator is the one of apply.cu / apply_fast.cu (one-body hops of both
// spins, the diagonal of Eq. 1 / Eq. 2 / the Sec. 4 Hamiltonian, spin-flip and
// pair-hopping).  The layout cuts memory instructions per matrix element:
//
//  * A block takes R up strings (rows) at a time, in the one-body-component
//    order of the fast tables (neighbour rows stay resident in L2), and stages
//    their x rows in shared memory interleaved, R elements per down rank, so
//    one vector load gathers a down-hop target for all R rows and one hop word
//    and one coefficient serve R rows.
//  * Lane l of a warp owns down string 32 g + l (natural order).  The gathers
//    of the up hops and spin-flip / pair-hop moves, the diagonal tables and the
//    stores are then whole lines per warp.  The down-hop lists are padded per
//    group of 32 strings to the group's longest list with a zero coefficient
//    on staged element 0 (a broadcast read).
//  * Each element is summed in two passes, in a fixed order:
//      A = diag * x + sum over down hops        (row-local, staged row)
//      B = sum over up hops, spin-flip, pair-hop (other rows, from L2)
//    and y = A + B rounded once.
//      float vectors: A and B are float sums (one FMA per term) with the
//        coefficients rounded to float and the diagonal formed in float from
//        three float pieces (e_up + e_dn + W), y = fl(A + B); with u = 2^-24,
//        n_A and n_B terms and S_i the summed magnitude of the density terms
//        behind the diagonal, |y - (Hx)_i| <= u [(n_A + 1) sum_A |H_ij x_j| +
//        4 S_i |x_i| + (n_B + 1) sum_B |H_ij x_j| + |(Hx)_i|] to first order.
//      double-float vectors: every product and sum in double-float (Dekker /
//        Knuth error-free transformations, about 2^-46 relative), A + B
//        normalised once.
//  * With the impurity orbitals on the top sites a spin-flip / pair-hop move
//    shifts a down rank by a constant per impurity pattern; the rows' term
//    lists per pattern hold their up hops, then the moves that apply to that
//    pattern with the shift folded into the element offset and the sign into
//    the coefficient.  A lane reads the list of its own string's pattern, so a
//    warp whose 32 strings share a pattern (all but a few) reads one list.
//    The R rows' lists of a pattern are padded to a common length with zero
//    terms on the row itself, so that one step serves all R rows; the
//    gathers of the first CH steps are issued before the down hops.
//
// Every variant (R, threads per block) adds the same terms in the same order
// (padding adds exact zeros), so the variants of one format agree bit for bit.
#include <algorithm>
#include <climits>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr int kMaxCoefN = 256;
constexpr int kMaxDeltaN = 256;
constexpr int kMaxPatN = 16;   // diagonal patterns (16 x 16 cross table)

struct NatF32 {
  using V = float;   // stored element
  using C = float;   // coefficient
  using A = float;   // accumulator
  __device__ static __forceinline__ A zero() { return 0.f; }
  __device__ static __forceinline__ C czero() { return 0.f; }
  __device__ static __forceinline__ void mac(A& a, C c, V x) { a = __fmaf_rn(c, x, a); }
  __device__ static __forceinline__ V fin(A a, A b) { return __fadd_rn(a, b); }
  __device__ static __forceinline__ void dot(float2& d, V x, V y) { df_mac1(d, make_float2(x, 0.f), y); }
};

struct NatDF {
  using V = float2;
  using C = float2;
  using A = float2;
  __device__ static __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ C czero() { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ void mac(A& a, C c, V x) { df_mac(a, c, x); }
  __device__ static __forceinline__ V fin(A a, A b) { return df_add(a, b); }
  __device__ static __forceinline__ void dot(float2& d, V x, V y) { df_mac(d, x, y); }
};

// R elements (or coefficients, or offsets) side by side, one vector access.
template <class T, int R>
struct alignas(sizeof(T) * R) Vec {
  T v[R];
};

struct NatView {
  uint32_t D_up, D, n_grp, max_cnt;
  const uint32_t* row_order;
  const uint32_t* row_pat;      // diagonal pattern of each up string
  const uint32_t* hop;          // [n_grp][max_cnt/2][32][2]: target rank << 8 | coefficient id (max_cnt even)
  const uint32_t* meta;         // [n_grp*32]: hop count | diagonal pattern << 8 | impurity pattern << 16
  const void* coef;             // [n_coef] down-hop coefficients (float or double-float)
  int n_coef;
  // diagonal, float: e_up[u] + e_dn[d] + W[pu][pd] in float; double-float:
  // dd[pu][d] = e_dn[d] + W[pu][pd] (from double) times x, plus e_up[u] times x
  const float* e_dn;            // [n_grp*32] (float)
  const float* W;               // [n_pat][n_pat] (float)
  const float2* dd;             // [n_pat][n_grp*32] (double-float)
  int n_pat;
  const double* e_up;
  const uint32_t *uh_ptr, *uh_tgt;
  const double* uh_val;
  const uint32_t *mx_ptr, *mx_tgt;
  const double* mx_val;
  const uint8_t* mx_mv;
  const int32_t* mdelta;        // [M*M][np]: (shift << 1 | sign) or INT_MIN; NULL without moves
  int np, n_md;
  int n_lp;                     // term lists per row (np with moves, else 1)
  uint32_t lcap;                // entries per list
  double* dotp;                 // optional per-block partial sums of <x, y>
};

__host__ __device__ inline size_t a16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared memory of one block; the kernel carves it in this order.
size_t nat_smem(int R, size_t vbytes, uint32_t D, int n_coef, int n_pat, int n_md, int n_lp, uint32_t lcap) {
  const size_t nl = (size_t)R * n_lp;
  return a16((size_t)D * vbytes * R) + a16((size_t)n_coef * vbytes) + a16((size_t)n_pat * n_pat * 4) +
         a16((size_t)n_md * 4) + a16(nl * lcap * 4) + a16(nl * lcap * vbytes) + a16(nl * 4) + a16((size_t)n_lp * 4) +
         a16((size_t)R * vbytes) + a16((size_t)R * 8);
}

template <class V>
__device__ __forceinline__ void cp_async_elem(V* s, const V* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(g), "n"(sizeof(V)));
}
__device__ __forceinline__ void cp_async_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <class P, int R, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_apply_nat(NatView F, const typename P::V* __restrict__ x,
                                                       typename P::V* __restrict__ y) {
  using V = typename P::V;
  using C = typename P::C;
  using A = typename P::A;
  using XV = Vec<V, R>;
  using OV = Vec<int, R>;
  using CV = Vec<C, R>;
  constexpr bool kF32 = sizeof(V) == 4;
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr int NWARP = BS / 32;
  static_assert(NWARP >= R, "one warp builds the term lists of each row");
  const uint32_t D = F.D;
  const uint32_t lcap = F.lcap;
  const int n_lp = F.n_lp;
  unsigned char* p = sm;
  XV* xs = reinterpret_cast<XV*>(p);              // staged rows, interleaved
  p += a16((size_t)D * sizeof(XV));
  C* cs = reinterpret_cast<C*>(p);                // down-hop coefficients
  p += a16((size_t)F.n_coef * sizeof(C));
  float* ws = reinterpret_cast<float*>(p);        // cross diagonal table (float vectors)
  p += a16((size_t)F.n_pat * F.n_pat * 4);
  int32_t* mds = reinterpret_cast<int32_t*>(p);   // move shifts per impurity pattern
  p += a16((size_t)F.n_md * 4);
  int* loff = reinterpret_cast<int*>(p);          // term lists [n_lp][lcap][R]: element offsets
  p += a16((size_t)R * n_lp * lcap * 4);
  C* lcf = reinterpret_cast<C*>(p);               // ... and coefficients
  p += a16((size_t)R * n_lp * lcap * sizeof(C));
  int* ln = reinterpret_cast<int*>(p);            // list lengths [R][n_lp]
  p += a16((size_t)R * n_lp * 4);
  int* lmx = reinterpret_cast<int*>(p);           // padded list length per pattern [n_lp]
  p += a16((size_t)n_lp * 4);
  C* eus = reinterpret_cast<C*>(p);               // e_up of each row
  p += a16((size_t)R * sizeof(C));
  int* pus = reinterpret_cast<int*>(p);           // diagonal pattern of each row
  int* urs = pus + R;                             // element offset u * D of each row
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr bool kDyn = MINB == 1;   // one block per SM: groups handed out on demand
  __shared__ uint32_t gnext;          // next group of the tile not yet taken

  const C* gcoef = static_cast<const C*>(F.coef);
  for (int k = threadIdx.x; k < F.n_coef; k += BS) cs[k] = gcoef[k];
  if (kF32)
    for (int k = threadIdx.x; k < F.n_pat * F.n_pat; k += BS) ws[k] = F.W[k];
  for (int k = threadIdx.x; k < F.n_md; k += BS) mds[k] = F.mdelta[k];
  float2 dacc = make_float2(0.f, 0.f);  // <x, y> over this thread's elements (only with F.dotp)
  const uint64_t NE = (uint64_t)F.n_grp * 32;

  const uint32_t n_tiles = (F.D_up + R - 1) / R;
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    __syncthreads();  // the previous tile is done with the staged rows and lists
    if (kDyn && threadIdx.x == 0) gnext = NWARP;   // groups past the warps' first ones go on demand
    {
      const V* xr[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = t * R + r;
        xr[r] = x + (uint64_t)F.row_order[i < F.D_up ? i : t * R] * D;
      }
      V* xf = reinterpret_cast<V*>(xs);
      for (uint32_t d = threadIdx.x; d < D; d += BS) {
#pragma unroll
        for (int r = 0; r < R; ++r) cp_async_elem(xf + (size_t)d * R + r, xr[r] + d);
      }
    }
    if (warp < R) {
      // warp r writes row r's entries of every pattern's list: the up hops,
      // then the moves that apply to that pattern (at most 64 of each per row);
      // entry k of row r in the list of pattern q sits at (q * lcap + k) * R + r
      const int r = warp;
      const bool vr = t * R + r < F.D_up;
      const uint32_t uu = F.row_order[vr ? t * R + r : t * R];
      const uint32_t h0 = F.uh_ptr[uu], nh = vr ? F.uh_ptr[uu + 1] - h0 : 0u;
      for (uint32_t k = lane; k < nh; k += 32) {
        const int off = (int)(F.uh_tgt[h0 + k] * D);
        const double v = F.uh_val[h0 + k];
        C c;
        if constexpr (kF32) c = (float)v;
        else c = df_from_double(v);
        for (int q = 0; q < n_lp; ++q) {
          loff[((size_t)q * lcap + k) * R + r] = off;
          lcf[((size_t)q * lcap + k) * R + r] = c;
        }
      }
      int cnt_q = (int)nh;  // lane q's list length (lanes < n_lp)
      if (F.mdelta && vr) {
        const uint32_t m0 = F.mx_ptr[uu], nmr = F.mx_ptr[uu + 1] - m0;
        const uint32_t ja = lane, jb = lane + 32;
        const bool va = ja < nmr, vb = jb < nmr;
        const int ta = va ? (int)(F.mx_tgt[m0 + ja] * D) : 0;
        const int tb = vb ? (int)(F.mx_tgt[m0 + jb] * D) : 0;
        const double ca = va ? F.mx_val[m0 + ja] : 0.0;
        const double cb = vb ? F.mx_val[m0 + jb] : 0.0;
        const uint32_t qa = va ? (uint32_t)F.mx_mv[m0 + ja] * (uint32_t)F.np : 0u;
        const uint32_t qb = vb ? (uint32_t)F.mx_mv[m0 + jb] * (uint32_t)F.np : 0u;
        const uint32_t below = (1u << lane) - 1u;
        for (int q = 0; q < n_lp; ++q) {
          const int32_t mda = va ? mds[qa + q] : INT_MIN, mdb = vb ? mds[qb + q] : INT_MIN;
          const unsigned ba = __ballot_sync(0xffffffffu, mda != INT_MIN);
          const unsigned bb = __ballot_sync(0xffffffffu, mdb != INT_MIN);
          const size_t base = (size_t)q * lcap + nh;
          if (mda != INT_MIN) {
            const size_t at = (base + __popc(ba & below)) * R + r;
            const double v = (mda & 1) ? -ca : ca;
            loff[at] = ta + (mda >> 1);
            if constexpr (kF32) lcf[at] = (float)v;
            else lcf[at] = df_from_double(v);
          }
          if (mdb != INT_MIN) {
            const size_t at = (base + __popc(ba) + __popc(bb & below)) * R + r;
            const double v = (mdb & 1) ? -cb : cb;
            loff[at] = tb + (mdb >> 1);
            if constexpr (kF32) lcf[at] = (float)v;
            else lcf[at] = df_from_double(v);
          }
          if (lane == q) cnt_q = (int)nh + __popc(ba) + __popc(bb);
        }
      }
      if (lane < n_lp) ln[r * n_lp + lane] = cnt_q;
      if (lane == 0) {
        if constexpr (kF32) eus[r] = (float)F.e_up[uu];
        else eus[r] = df_from_double(F.e_up[uu]);
        pus[r] = (int)F.row_pat[uu];
        urs[r] = (int)(uu * D);
      }
    }
    __syncthreads();
    // the rows of a pattern's list share one length: shorter rows are padded
    // with zero-coefficient terms on their own row
    for (int q = threadIdx.x; q < n_lp; q += BS) {
      int m = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) m = max(m, ln[r * n_lp + q]);
      lmx[q] = m;
    }
    for (int idx = threadIdx.x; idx < n_lp * (int)lcap * R; idx += BS) {
      const int r = idx % R, k = (idx / R) % (int)lcap, q = idx / (R * (int)lcap);
      if (k < ln[r * n_lp + q]) continue;
      int m = 0;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) m = max(m, ln[rr * n_lp + q]);
      if (k < m) {
        loff[idx] = urs[r];
        lcf[idx] = P::czero();
      }
    }
    cp_async_all();
    __syncthreads();

    // With one block per SM each warp takes group `warp` first, then the next
    // untaken one, so the warps end a tile together however the groups' costs
    // vary (N_s = 16, four rows, 1024 x 1: 1.29 ms against 1.50 ms with every
    // NWARP-th group); with two blocks per SM the other block fills the tail
    // of a tile and the fixed order reads neighbouring groups together.
    auto next_group = [&](uint32_t g) {
      if constexpr (!kDyn) {
        return g + NWARP;
      } else {
        uint32_t nx = 0;
        if (lane == 0) nx = atomicAdd(&gnext, 1u);
        return __shfl_sync(0xffffffffu, nx, 0);
      }
    };
    for (uint32_t g = warp; g < F.n_grp; g = next_group(g)) {
      const uint32_t d = g * 32 + lane;
      const bool ok = d < D;
      const uint32_t mt = __ldg(F.meta + d);   // padding entries: count 0, patterns 0
      const int cnt = (int)(mt & 255u);
      const int pd = (int)((mt >> 8) & 255u);
      const int ip = (int)(mt >> 16);
      const XV xv = xs[ok ? d : 0u];
      A Aa[R], Bb[R];
      if constexpr (kF32) {
        const float edn = __ldg(F.e_dn + d);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float dg = __fadd_rn(__fadd_rn(eus[r], edn), ws[pus[r] * F.n_pat + pd]);
          Aa[r] = __fmul_rn(dg, xv.v[r]);
          Bb[r] = P::zero();
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const C dg = __ldg(F.dd + (uint64_t)pus[r] * NE + d);
          Aa[r] = P::zero();
          P::mac(Aa[r], dg, xv.v[r]);
          P::mac(Aa[r], eus[r], xv.v[r]);
          Bb[r] = P::zero();
        }
      }
      // pass B set-up: this string's pattern list, all R rows per step.  The
      // gathers of its first CH steps are issued now, so that their L2
      // latency overlaps the shared-memory work of the down hops.
      constexpr int CH = kF32 ? 16 / R : 4;   // float: 16 gathers in flight per thread
      const int nl = ok ? lmx[ip] : 0;
      const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)nl);
      const OV* Lo = reinterpret_cast<const OV*>(loff + (size_t)ip * lcap * R);
      const CV* Lc = reinterpret_cast<const CV*>(lcf + (size_t)ip * lcap * R);
      const V* xd = x + d;
      V xc[CH][R];
      // A chunk whose CH steps all lie in this lane's list runs without the
      // per-step guards.
      auto gather = [&](int k0) {
        if (k0 + CH <= nl) {
#pragma unroll
          for (int s = 0; s < CH; ++s) {
            const OV o = Lo[k0 + s];
#pragma unroll
            for (int r = 0; r < R; ++r) xc[s][r] = __ldg(xd + o.v[r]);
          }
        } else {
#pragma unroll
          for (int s = 0; s < CH; ++s) {
            if (k0 + s < nl) {
              const OV o = Lo[k0 + s];
#pragma unroll
              for (int r = 0; r < R; ++r) xc[s][r] = __ldg(xd + o.v[r]);
            }
          }
        }
      };
      auto add = [&](int k0) {
        if (k0 + CH <= nl) {
#pragma unroll
          for (int s = 0; s < CH; ++s) {
            const CV c = Lc[k0 + s];
#pragma unroll
            for (int r = 0; r < R; ++r) P::mac(Bb[r], c.v[r], xc[s][r]);
          }
        } else {
#pragma unroll
          for (int s = 0; s < CH; ++s) {
            if (k0 + s < nl) {
              const CV c = Lc[k0 + s];
#pragma unroll
              for (int r = 0; r < R; ++r) P::mac(Bb[r], c.v[r], xc[s][r]);
            }
          }
        }
      };
      gather(0);
      // pass A: down hops of the staged rows, padded to the group's longest
      // list; hop words four at a time (two 8-byte loads: a string's hops 2j
      // and 2j + 1 sit side by side), the next four loaded ahead
      {
        const int gm = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
        const uint2* hp = reinterpret_cast<const uint2*>(F.hop) + (size_t)g * (F.max_cnt / 2) * 32 + lane;
        uint2 h[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) h[i] = 2 * i < gm ? __ldg(hp + (size_t)i * 32) : make_uint2(0u, 0u);
        for (int k = 0; k < gm; k += 4) {
          uint2 hn[2];
#pragma unroll
          for (int i = 0; i < 2; ++i)
            hn[i] = k + 4 + 2 * i < gm ? __ldg(hp + (size_t)((k + 4) / 2 + i) * 32) : make_uint2(0u, 0u);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (k + i < gm) {
              const uint32_t wd = (i & 1) ? h[i >> 1].y : h[i >> 1].x;
              const C c = cs[wd & 255u];
              const XV X = xs[wd >> 8];
#pragma unroll
              for (int r = 0; r < R; ++r) P::mac(Aa[r], c, X.v[r]);
            }
          }
#pragma unroll
          for (int i = 0; i < 2; ++i) h[i] = hn[i];
        }
      }
      // pass B: CH steps per round trip
      add(0);
      for (int k0 = CH; k0 < nmax; k0 += CH) {
        gather(k0);
        add(k0);
      }
      if (ok) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (t * R + r >= F.D_up) continue;
          const V yv = P::fin(Aa[r], Bb[r]);
          __stcs(y + (uint32_t)urs[r] + d, yv);
          if (F.dotp) P::dot(dacc, xv.v[r], yv);
        }
      }
    }
  }
  if (F.dotp) {
    __shared__ float2 red[NWARP];
    for (int o = 16; o > 0; o >>= 1)
      dacc = df_add(dacc, make_float2(__shfl_xor_sync(0xffffffffu, dacc.x, o), __shfl_xor_sync(0xffffffffu, dacc.y, o)));
    if (lane == 0) red[warp] = dacc;
    __syncthreads();
    if (warp == 0) {
      float2 v = lane < NWARP ? red[lane] : make_float2(0.f, 0.f);
      for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
      if (lane == 0) F.dotp[blockIdx.x] = (double)v.x + (double)v.y;
    }
  }
}

// Natural-order tables, one thread per down string (padding strings up to the
// group boundary get count 0 and patterns 0).  With dd != NULL also the
// double-float diagonal rows dd[pu][d] = e_dn[d] + W[pu][pd(d)] for every up
// pattern pu.
__global__ void k_nat_tables(uint32_t D, uint32_t n_grp, uint32_t max_cnt, const uint32_t* __restrict__ dbasis,
                             const uint32_t* __restrict__ dh_ptr, const uint32_t* __restrict__ dh_tgt,
                             const double* __restrict__ dh_val, const double* __restrict__ coef, int n_coef,
                             int zero_id, const double* __restrict__ e_dn, const double* __restrict__ W, int w_lo,
                             int wbits, int orb0, int M, uint32_t* __restrict__ hop, uint32_t* __restrict__ meta,
                             float* __restrict__ edn, float2* __restrict__ dd) {
  const uint32_t d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_grp * 32) return;
  const uint32_t g = d / 32, lane = d % 32;
  const bool real = d < D;
  const uint32_t h0 = real ? dh_ptr[d] : 0u, c = real ? dh_ptr[d + 1] - h0 : 0u;
  for (uint32_t k = 0; k < max_cnt; ++k) {  // max_cnt even: hops 2j, 2j + 1 side by side
    uint32_t word = (uint32_t)zero_id;  // staged element 0 times the zero coefficient
    if (k < c) {
      const double v = dh_val[h0 + k];
      int id = 0;
      while (id < n_coef && coef[id] != v) ++id;
      word = (dh_tgt[h0 + k] << 8) | (uint32_t)id;
    }
    hop[(((size_t)g * (max_cnt / 2) + k / 2) * 32 + lane) * 2 + (k & 1)] = word;
  }
  const uint32_t s = real ? dbasis[d] : 0u;
  const uint32_t pd = (real && wbits > 0) ? ((s >> w_lo) & ((1u << wbits) - 1u)) : 0u;
  const uint32_t ip = (real && M > 0) ? ((s >> orb0) & ((1u << M) - 1u)) : 0u;
  meta[d] = c | (pd << 8) | (ip << 16);
  edn[d] = real ? (float)e_dn[d] : 0.f;
  if (dd) {
    const uint64_t NE = (uint64_t)n_grp * 32;
    for (uint32_t pu = 0; pu < (1u << wbits); ++pu) {
      double v = 0.0;
      if (real) {
        v = e_dn[d];
        if (W) v += W[(pu << wbits) + pd];
      }
      dd[pu * NE + d] = df_from_double(v);
    }
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

NatView make_nat_view(const Sector* s) {
  const auto& f = s->fast;
  NatView F;
  F.D_up = s->up.D;
  F.D = s->dn.D;
  F.n_grp = f.nat_grp;
  F.max_cnt = f.nat_mc;
  F.row_order = f.row_order;
  F.row_pat = f.row_pat;
  F.hop = f.nat_hop;
  F.meta = f.nat_meta;
  F.coef = s->prec == ED_PREC_FP32 ? (const void*)f.nat_coef : (const void*)f.coef_df;
  F.n_coef = f.n_coef;
  F.e_dn = f.nat_edn;
  F.W = f.nat_W;
  F.dd = f.nat_dd;
  F.n_pat = f.n_pat;
  F.e_up = s->up.e;
  F.uh_ptr = s->up.hop_ptr;
  F.uh_tgt = s->up.hop_tgt;
  F.uh_val = s->up.hop_val;
  F.mx_ptr = s->mx_ptr;
  F.mx_tgt = s->mx_tgt;
  F.mx_val = s->mx_val;
  F.mx_mv = s->mx_mv;
  F.mdelta = f.mix_delta ? f.mdelta : nullptr;
  F.np = 1 << s->M;
  F.n_md = f.mix_delta ? s->M * s->M * (1 << s->M) : 0;
  F.n_lp = f.n_lp;
  F.lcap = f.lcap;
  F.dotp = nullptr;
  return F;
}

template <class P, int R, int BS, int MINB>
int launch_nat_t(const Sector* s, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts) {
  using V = typename P::V;
  NatView F = make_nat_view(s);
  F.dotp = dotp;
  const size_t smem = nat_smem(R, sizeof(V), F.D, F.n_coef, F.n_pat, F.n_md, F.n_lp, F.lcap);
  auto kern = k_apply_nat<P, R, BS, MINB>;
  ED_TRY(smem_cap(s->ctx, kern, smem));
  int per_sm = 0;
  ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem));
  if (per_sm < 1) ED_INVALID("natural-order kernel does not fit on an SM (%zu B shared)", smem);
  const uint32_t n_tiles = (F.D_up + R - 1) / R;
  const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)s->ctx->num_sms * per_sm, n_tiles);
  kern<<<grid, BS, smem, st>>>(F, static_cast<const V*>(x), static_cast<V*>(y));
  ED_LAUNCH_CHECK();
  if (nparts) *nparts = (int)grid;
  return ED_OK;
}

// Variants per format: rows per block R x threads per block x blocks per SM
// the register budget is sized for (shared memory may allow fewer).
constexpr int kNatR[2][kNatVariants] = {{4, 4, 4, 2, 2, 2}, {2, 2, 2, 1, 1, 1}};
constexpr int kNatBS[2][kNatVariants] = {{1024, 512, 384, 256, 512, 384}, {256, 512, 384, 256, 512, 384}};
constexpr int kNatMinB[2][kNatVariants] = {{1, 2, 2, 3, 2, 2}, {2, 1, 2, 3, 2, 2}};

int fmt_of(int prec) { return prec == ED_PREC_FP32 ? 0 : 1; }
int fmt_of(const Sector* s) { return fmt_of(s->prec); }

}  // namespace

void nat_variant_info(int prec, int v, int* rows, int* block, int* min_blocks) {
  const int f = fmt_of(prec);
  *rows = kNatR[f][v];
  *block = kNatBS[f][v];
  *min_blocks = kNatMinB[f][v];
}

size_t nat_variant_smem(const Sector* s, int v) {
  const auto& f = s->fast;
  return nat_smem(kNatR[fmt_of(s)][v], elem_bytes(s->prec), s->dn.D, f.n_coef, f.n_pat,
                  f.mix_delta ? s->M * s->M * (1 << s->M) : 0, f.n_lp, f.lcap);
}

int launch_nat(const Sector* s, int v, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts) {
  if (!s->fast.nat_ok) ED_INVALID("the sector has no natural-order tables");
  if (s->prec == ED_PREC_FP32) {
    switch (v) {
      case 0: return launch_nat_t<NatF32, 4, 1024, 1>(s, x, y, st, dotp, nparts);
      case 1: return launch_nat_t<NatF32, 4, 512, 2>(s, x, y, st, dotp, nparts);
      case 2: return launch_nat_t<NatF32, 4, 384, 2>(s, x, y, st, dotp, nparts);
      case 3: return launch_nat_t<NatF32, 2, 256, 3>(s, x, y, st, dotp, nparts);
      case 4: return launch_nat_t<NatF32, 2, 512, 2>(s, x, y, st, dotp, nparts);
      case 5: return launch_nat_t<NatF32, 2, 384, 2>(s, x, y, st, dotp, nparts);
    }
  } else if (s->prec == ED_PREC_DF64) {
    switch (v) {
      case 0: return launch_nat_t<NatDF, 2, 256, 2>(s, x, y, st, dotp, nparts);
      case 1: return launch_nat_t<NatDF, 2, 512, 1>(s, x, y, st, dotp, nparts);
      case 2: return launch_nat_t<NatDF, 2, 384, 2>(s, x, y, st, dotp, nparts);
      case 3: return launch_nat_t<NatDF, 1, 256, 3>(s, x, y, st, dotp, nparts);
      case 4: return launch_nat_t<NatDF, 1, 512, 2>(s, x, y, st, dotp, nparts);
      case 5: return launch_nat_t<NatDF, 1, 384, 2>(s, x, y, st, dotp, nparts);
    }
  }
  ED_INVALID("natural-order variant %d does not apply", v);
}

// Tables of the natural-order kernel for float and double-float sectors;
// leaves nat_ok false where it does not apply (moves without the top-site
// shift layout, a cross diagonal table over more than 4 sites, rows too long
// for shared memory).
int build_nat(Sector* s, const std::vector<double>& coef, int zero_id) {
  auto& f = s->fast;
  f.nat_ok = false;
  if ((s->prec != ED_PREC_FP32 && s->prec != ED_PREC_DF64) || !f.ok) return ED_OK;
  if (s->prec == ED_PREC_FP32 && s->acc_df) return ED_OK;  // the caller keeps double-float sums
  if (s->n_mix && !f.mix_delta) return ED_OK;
  if (f.n_pat > kMaxPatN || (int)coef.size() > kMaxCoefN) return ED_OK;
  if (f.mix_delta && s->M * s->M * (1 << s->M) > kMaxDeltaN) return ED_OK;
  const uint32_t D = s->dn.D;
  if (D >= (1u << 24) || s->dim >= (1ull << 31)) return ED_OK;
  const int rmin = s->prec == ED_PREC_FP32 ? 2 : 1;
  if (nat_smem(rmin, elem_bytes(s->prec), D, (int)coef.size(), f.n_pat,
               f.mix_delta ? s->M * s->M * (1 << s->M) : 0, f.n_lp, f.lcap) > 220 * 1024)
    return ED_OK;
  const uint32_t n_grp = (D + 31) / 32;
  f.nat_grp = n_grp;
  f.nat_mc = (f.max_cnt + 1) & ~1u;
  const uint64_t NE = (uint64_t)n_grp * 32;
  ED_TRY(sector_alloc(s, &f.nat_hop, (size_t)f.nat_mc * NE));
  ED_TRY(sector_alloc(s, &f.nat_meta, NE));
  ED_TRY(sector_alloc(s, &f.nat_edn, NE));
  ED_TRY(sector_alloc(s, &f.nat_coef, coef.size()));
  ED_TRY(sector_alloc(s, &f.nat_W, (size_t)f.n_pat * f.n_pat));
  if (s->prec == ED_PREC_DF64) ED_TRY(sector_alloc(s, &f.nat_dd, (size_t)f.n_pat * NE));
  const int wbits = (s->n_chunks == 1) ? s->w_bits[0] : 0;
  const double* W = (s->n_chunks == 1) ? s->W : nullptr;
  k_nat_tables<<<(unsigned)((NE + 127) / 128), 128>>>(
      D, n_grp, f.nat_mc, s->dn.basis, s->dn.hop_ptr, s->dn.hop_tgt, s->dn.hop_val, f.coef, (int)coef.size(), zero_id,
      s->dn.e, W, s->w_lo, wbits, s->orb0, f.mix_delta ? s->M : 0, f.nat_hop, f.nat_meta, f.nat_edn,
      s->prec == ED_PREC_DF64 ? f.nat_dd : nullptr);
  ED_LAUNCH_CHECK();
  k_to_f32<<<(unsigned)((coef.size() + 127) / 128), 128>>>(f.coef, f.nat_coef, (uint32_t)coef.size());
  ED_LAUNCH_CHECK();
  // cross diagonal table W[pu][pd] of the single chunk (all zero without one)
  const uint32_t nw = (uint32_t)f.n_pat * f.n_pat;
  if (W) {
    k_to_f32<<<(nw + 127) / 128, 128>>>(W, f.nat_W, nw);
    ED_LAUNCH_CHECK();
  } else {
    ED_TRY_CUDA(cudaMemset(f.nat_W, 0, sizeof(float) * nw));
  }
  ED_TRY_CUDA(cudaStreamSynchronize(0));
  f.nat_ok = true;
  return ED_OK;
}

}  // namespace ed
