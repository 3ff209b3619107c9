// Matrix-free sector H*v (the "evaluate the matrix elements whenever needed"
// improvement named at the end of Sec. 3.2), fused in one pass per element:
//
//   y[u,d] = diag(u,d) x[u,d]                                  diagonal (Eq. 1, 2, Sec. 4)
//          + sum_{d' in hops(d)} t x[u,d']                      down-spin one-body hops
//          + sum_{u' in hops(u)} t x[u',d]                      up-spin one-body hops
//          + sum_{(u'',mv) in mix(u)} J' s_u s_d x[u'',mv(d)]   spin-flip / pair-hop (Sec. 4)
//
// diag(u,d) = e_up[u] + e_dn[d] + sum_c W_c[u_c][d_c].
// Two launch shapes share the per-element code and summation order (so they
// give bit-identical results): a flat grid (thread per element, rows read from
// L1/L2) for short rows, and a row-staged persistent kernel (one up-string row
// of x staged in shared memory per block iteration) for long rows.
#include <algorithm>

#include "apply_common.h"

namespace ed {

namespace {

// Flat launch: blockIdx.y walks up rows, x-dimension covers the row.
template <class P>
__global__ void __launch_bounds__(256) k_apply_flat(SectorView S, const uint32_t* __restrict__ ub,
                                                    const uint32_t* __restrict__ db,
                                                    const typename P::V* __restrict__ x,
                                                    typename P::V* __restrict__ y) {
  const uint32_t Dd = S.D_dn;
  uint32_t d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= Dd) return;
  uint32_t sd = db[d];
  for (uint32_t u = blockIdx.y; u < S.D_up; u += gridDim.y) {
    const typename P::V* xr = x + (uint64_t)u * Dd;
    auto xrow = [xr](uint32_t j) { return xr[j]; };
    y[(uint64_t)u * Dd + d] = element<P>(S, x, u, ub[u], d, sd, row_e<P>(S, u), xrow);
  }
}

// Row-staged persistent launch: one up row at a time per block, x row in smem.
template <class P>
__global__ void __launch_bounds__(256) k_apply_rows(SectorView S, const uint32_t* __restrict__ ub,
                                                    const uint32_t* __restrict__ db,
                                                    const typename P::V* __restrict__ x,
                                                    typename P::V* __restrict__ y) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);
  const uint32_t Dd = S.D_dn;
  for (uint32_t u = blockIdx.x; u < S.D_up; u += gridDim.x) {
    __syncthreads();
    const V* xr = x + (uint64_t)u * Dd;
    for (uint32_t j = threadIdx.x; j < Dd; j += blockDim.x) xs[j] = xr[j];
    __syncthreads();
    const uint32_t su = ub[u];
    const typename P::C eu = row_e<P>(S, u);
    auto xrow = [xs](uint32_t j) { return xs[j]; };
    V* yr = y + (uint64_t)u * Dd;
    for (uint32_t d = threadIdx.x; d < Dd; d += blockDim.x)
      yr[d] = element<P>(S, x, u, su, d, db[d], eu, xrow);
  }
}

template <class P>
int launch(const Sector* s, const void* xv, void* yv, cudaStream_t st) {
  using V = typename P::V;
  SectorView S = s->view();
  const V* x = static_cast<const V*>(xv);
  V* y = static_cast<V*>(yv);
  const uint32_t Dd = S.D_dn, Du = S.D_up;
  size_t row_bytes = (size_t)Dd * sizeof(V);
  const Ctx* c = s->ctx;
  if (Dd >= 1024 && row_bytes <= 96 * 1024) {
    static bool attr_set = false;  // per policy instantiation
    if (!attr_set) {
      ED_TRY_CUDA(cudaFuncSetAttribute(k_apply_rows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       96 * 1024));
      attr_set = true;
    }
    int per_sm = 0;
    ED_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_rows<P>, 256, row_bytes));
    if (per_sm < 1) per_sm = 1;
    uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)c->num_sms * per_sm, Du);
    k_apply_rows<P><<<grid, 256, row_bytes, st>>>(S, s->up.basis, s->dn.basis, x, y);
  } else {
    dim3 grid((Dd + 255) / 256, std::min<uint32_t>(Du, 65535u));
    k_apply_flat<P><<<grid, 256, 0, st>>>(S, s->up.basis, s->dn.basis, x, y);
  }
  ED_LAUNCH_CHECK();
  return ED_OK;
}

}  // namespace

int apply_h(const Sector* s, const void* x, void* y, cudaStream_t st) {
  if (!x || !y) ED_INVALID("x or y is NULL");
  if (x == y) ED_INVALID("x and y must not overlap");
  if (s->fast.ok) return apply_fast(s, x, y, st);
  switch (s->prec) {
    case ED_PREC_FP64: return launch<PolF64>(s, x, y, st);
    case ED_PREC_DF64: return launch<PolDF>(s, x, y, st);
    case ED_PREC_FP32: return launch<PolF32>(s, x, y, st);
  }
  ED_INVALID("unknown precision");
}

}  // namespace ed
