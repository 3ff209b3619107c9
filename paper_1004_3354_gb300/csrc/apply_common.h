// Per-element evaluation of the matrix-free H*v shared by the generic apply
// kernels and the batched multi-sector kernels (internal header).
#pragma once

#include "ed_internal.h"

namespace ed {

// Diagonal contribution.  FP64 forms diag in double and multiplies once;
// the double-float policies multiply-accumulate each piece exactly.
template <class P>
struct Diag;

template <>
struct Diag<PolF64> {
  __device__ static __forceinline__ void apply(double& acc, const SectorView& S, uint32_t su, uint32_t d,
                                               uint32_t sd, double eu, double x) {
    double dg = eu + S.e_dn[d];
    for (int c = 0; c < S.n_chunks; ++c) {
      uint32_t uc = (su >> (S.w_lo + 8 * c)) & ((1u << S.w_bits[c]) - 1u);
      uint32_t dc = (sd >> (S.w_lo + 8 * c)) & ((1u << S.w_bits[c]) - 1u);
      dg += S.W[S.w_off[c] + (uc << S.w_bits[c]) + dc];
    }
    acc = fma(dg, x, acc);
  }
};

template <class P>
struct DiagDF {
  __device__ static __forceinline__ void apply(typename P::A& acc, const SectorView& S, uint32_t su,
                                               uint32_t d, uint32_t sd, float2 eu, typename P::V x) {
    P::mac(acc, eu, x);
    P::mac(acc, S.e_dn_df[d], x);
    for (int c = 0; c < S.n_chunks; ++c) {
      uint32_t uc = (su >> (S.w_lo + 8 * c)) & ((1u << S.w_bits[c]) - 1u);
      uint32_t dc = (sd >> (S.w_lo + 8 * c)) & ((1u << S.w_bits[c]) - 1u);
      P::mac(acc, S.W_df[S.w_off[c] + (uc << S.w_bits[c]) + dc], x);
    }
  }
};
template <>
struct Diag<PolDF> : DiagDF<PolDF> {};
template <>
struct Diag<PolF32> : DiagDF<PolF32> {};

template <class P>
__device__ __forceinline__ typename P::C row_e(const SectorView& S, uint32_t u);
template <>
__device__ __forceinline__ double row_e<PolF64>(const SectorView& S, uint32_t u) { return S.e_up[u]; }
template <>
__device__ __forceinline__ float2 row_e<PolDF>(const SectorView& S, uint32_t u) { return S.e_up_df[u]; }
template <>
__device__ __forceinline__ float2 row_e<PolF32>(const SectorView& S, uint32_t u) { return S.e_up_df[u]; }

// One output element.  u, d are ranks; su, sd the basis strings (the cross
// tables W are indexed by site occupations).
template <class P, class XRow>
__device__ __forceinline__ typename P::V element(const SectorView& S, const typename P::V* __restrict__ x,
                                                 uint32_t u, uint32_t su, uint32_t d, uint32_t sd,
                                                 typename P::C eu, XRow xrow) {
  using A = typename P::A;
  const uint32_t Dd = S.D_dn;
  A acc = P::zero();
  Diag<P>::apply(acc, S, su, d, sd, eu, xrow(d));
  // down-spin hops within the row
  for (uint32_t k = S.dh_ptr[d], e = S.dh_ptr[d + 1]; k < e; ++k)
    P::mac(acc, P::ld(S.dh_val, S.dh_val_df, k), xrow(S.dh_tgt[k]));
  // up-spin hops: same column of other rows
  for (uint32_t k = S.uh_ptr[u], e = S.uh_ptr[u + 1]; k < e; ++k)
    P::mac(acc, P::ld(S.uh_val, S.uh_val_df, k), x[(uint64_t)S.uh_tgt[k] * Dd + d]);
  // spin-flip and pair-hopping
  if (S.mx_ptr) {
    for (uint32_t k = S.mx_ptr[u], e = S.mx_ptr[u + 1]; k < e; ++k) {
      int32_t mv = S.dn_move[(uint32_t)S.mx_mv[k] * Dd + d];
      if (mv >= 0) {
        typename P::C c = P::ld(S.mx_val, S.mx_val_df, k);
        if (mv & 1) c = P::neg(c);
        P::mac(acc, c, x[(uint64_t)S.mx_tgt[k] * Dd + (uint32_t)(mv >> 1)]);
      }
    }
  }
  return P::out(acc);
}

}  // namespace ed
