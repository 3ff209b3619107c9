// Stored-CSR comparison variant: builds the sector Hamiltonian in the CSR
// layout of Fig. 1 (row start offsets, column of every stored entry, values;
// columns ascending within a row, the diagonal always stored, exact zeros
// omitted) and multiplies it by a vector as Listing 1 does (every row sums its
// stored entries times the vector at their columns).
#include <algorithm>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr int kRowMax = 512;

__device__ __forceinline__ double diag_f64(const SectorView& S, uint32_t u, uint32_t su, uint32_t d,
                                           uint32_t sd) {
  double dg = S.e_up[u] + S.e_dn[d];
  for (int c = 0; c < S.n_chunks; ++c) {
    uint32_t uc = (su >> (S.w_lo + 8 * c)) & ((1u << S.w_bits[c]) - 1u);
    uint32_t dc = (sd >> (S.w_lo + 8 * c)) & ((1u << S.w_bits[c]) - 1u);
    dg += S.W[S.w_off[c] + (uc << S.w_bits[c]) + dc];
  }
  return dg;
}

__global__ void k_csr_count(SectorView S, uint64_t* __restrict__ cnt) {
  uint64_t n = (uint64_t)S.D_up * S.D_dn;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u = (uint32_t)(i / S.D_dn), d = (uint32_t)(i % S.D_dn);
    uint64_t c = 1 + (S.dh_ptr[d + 1] - S.dh_ptr[d]) + (S.uh_ptr[u + 1] - S.uh_ptr[u]);
    if (S.mx_ptr)
      for (uint32_t k = S.mx_ptr[u]; k < S.mx_ptr[u + 1]; ++k)
        if (S.dn_move[(uint32_t)S.mx_mv[k] * S.D_dn + d] >= 0) ++c;
    cnt[i] = c;
  }
}

__global__ void k_csr_fill(SectorView S, const uint32_t* __restrict__ ub, const uint32_t* __restrict__ db,
                           const uint64_t* __restrict__ ptr, uint32_t* __restrict__ col,
                           double* __restrict__ val) {
  uint64_t n = (uint64_t)S.D_up * S.D_dn;
  uint32_t cc[kRowMax];
  double vv[kRowMax];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u = (uint32_t)(i / S.D_dn), d = (uint32_t)(i % S.D_dn);
    int m = 0;
    auto push = [&](uint32_t c, double v) {
      int k = m++;
      while (k > 0 && cc[k - 1] > c) {
        cc[k] = cc[k - 1];
        vv[k] = vv[k - 1];
        --k;
      }
      cc[k] = c;
      vv[k] = v;
    };
    push((uint32_t)i, diag_f64(S, u, ub[u], d, db[d]));
    for (uint32_t k = S.dh_ptr[d]; k < S.dh_ptr[d + 1]; ++k)
      push(u * S.D_dn + S.dh_tgt[k], S.dh_val[k]);
    for (uint32_t k = S.uh_ptr[u]; k < S.uh_ptr[u + 1]; ++k)
      push(S.uh_tgt[k] * S.D_dn + d, S.uh_val[k]);
    if (S.mx_ptr)
      for (uint32_t k = S.mx_ptr[u]; k < S.mx_ptr[u + 1]; ++k) {
        int32_t mv = S.dn_move[(uint32_t)S.mx_mv[k] * S.D_dn + d];
        if (mv >= 0) push(S.mx_tgt[k] * S.D_dn + (uint32_t)(mv >> 1), (mv & 1) ? -S.mx_val[k] : S.mx_val[k]);
      }
    uint64_t o = ptr[i];
    for (int k = 0; k < m; ++k) {
      col[o + k] = cc[k];
      val[o + k] = vv[k];
    }
  }
}

// Exclusive scan in place, 1024 elements per block; block totals to sums.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint64_t* __restrict__ a, uint64_t n,
                                                      uint64_t* __restrict__ sums) {
  __shared__ uint64_t wt[32];
  uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
  uint64_t v = (i < n) ? a[i] : 0;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t z = wt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t t = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += t;
    }
    wt[lane] = z;
  }
  __syncthreads();
  uint64_t incl = x + (w ? wt[w - 1] : 0);
  if (i < n) a[i] = incl - v;
  if (threadIdx.x == 1023) sums[blockIdx.x] = incl;
}

__global__ void k_scan_add(uint64_t* __restrict__ a, uint64_t n, const uint64_t* __restrict__ offs) {
  uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) a[i] += offs[blockIdx.x];
}

int scan_exclusive(Ctx* c, uint64_t* a, uint64_t n) {
  uint64_t nb = (n + 1023) / 1024;
  uint64_t* sums = nullptr;
  ED_TRY(dev_alloc_n(c, &sums, nb));
  k_scan_blocks<<<(uint32_t)nb, 1024>>>(a, n, sums);
  cudaError_t e = cudaGetLastError();
  int st = ED_OK;
  if (e == cudaSuccess && nb > 1) {
    st = scan_exclusive(c, sums, nb);
    if (st == ED_OK) {
      k_scan_add<<<(uint32_t)nb, 1024>>>(a, n, sums);
      e = cudaGetLastError();
    }
  }
  cudaError_t e2 = cudaDeviceSynchronize();
  dev_free(c, sums, nb * sizeof(uint64_t));
  if (st != ED_OK) return st;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    set_error("scan failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return ED_ERR_CUDA;
  }
  return ED_OK;
}

// Listing 1, LANES threads per row with a shuffle reduction.
template <int LANES>
__global__ void __launch_bounds__(256) k_csr_spmv(uint64_t nrows, const uint64_t* __restrict__ ptr,
                                                  const uint32_t* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ x, double* __restrict__ y) {
  uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x / LANES;
  int lane = threadIdx.x % LANES;
  for (uint64_t row = t / LANES; row < nrows; row += stride) {
    double acc = 0.0;
    for (uint64_t j = ptr[row] + lane; j < ptr[row + 1]; j += LANES) acc = fma(val[j], x[col[j]], acc);
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, LANES);
    if (lane == 0) y[row] = acc;
  }
}

}  // namespace

int build_csr(Sector* s) {
  if (s->prec != ED_PREC_FP64) ED_INVALID("the stored CSR variant is FP64 only");
  if (s->dim >= 0xffffffffull) ED_INVALID("sector too large for 32-bit CSR columns");
  uint64_t row_max = 1 + (uint64_t)s->up.max_hops + s->dn.max_hops + s->max_mix;
  if (row_max > (uint64_t)kRowMax) ED_INVALID("row too long for the CSR builder");
  Ctx* c = s->ctx;
  SectorView S = s->view();
  ED_TRY(sector_alloc(s, &s->csr_ptr, s->dim + 1));
  uint32_t grid = (uint32_t)std::min<uint64_t>((s->dim + 255) / 256, (uint64_t)c->num_sms * 16);
  ED_TRY_CUDA(cudaMemset(s->csr_ptr, 0, (s->dim + 1) * sizeof(uint64_t)));
  k_csr_count<<<grid, 256>>>(S, s->csr_ptr);
  ED_LAUNCH_CHECK();
  ED_TRY(scan_exclusive(c, s->csr_ptr, s->dim + 1));
  ED_TRY_CUDA(cudaMemcpy(&s->csr_nnz, s->csr_ptr + s->dim, sizeof(uint64_t), cudaMemcpyDeviceToHost));
  ED_TRY(sector_alloc(s, &s->csr_col, s->csr_nnz));
  ED_TRY(sector_alloc(s, &s->csr_val, s->csr_nnz));
  k_csr_fill<<<grid, 128>>>(S, s->up.basis, s->dn.basis, s->csr_ptr, s->csr_col, s->csr_val);
  ED_LAUNCH_CHECK();
  ED_TRY_CUDA(cudaStreamSynchronize(0));  // legacy stream only: leaves other work running
  return ED_OK;
}

int apply_h_csr(const Sector* s, const void* x, void* y, cudaStream_t st) {
  if (!s->csr_ptr) ED_INVALID("sector was created without ED_SECTOR_CSR");
  if (!x || !y || x == y) ED_INVALID("bad x / y");
  uint32_t grid = (uint32_t)std::min<uint64_t>((s->dim * 8 + 255) / 256, (uint64_t)s->ctx->num_sms * 32);
  if (grid == 0) grid = 1;
  k_csr_spmv<8><<<grid, 256, 0, st>>>(s->dim, s->csr_ptr, s->csr_col, s->csr_val,
                                      static_cast<const double*>(x), static_cast<double*>(y));
  ED_LAUNCH_CHECK();
  return ED_OK;
}

}  // namespace ed
