// C ABI entry points of libedgb (declared in include/ed.h): argument checks,
// handle ownership and error reporting around the device code.
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <new>
#include <string>

#include "ed_internal.h"

struct ed_ctx {
  ed::Ctx c;
};
struct ed_sector {
  ed::Sector s;
  ed::HostXfer* xfer = nullptr;  // buffers of ed_apply_h_host, made at its first call
};

namespace ed {

namespace {
thread_local std::string g_err;
}

Ctx* ctx_of(ed_ctx* h) { return h ? &h->c : nullptr; }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int dev_alloc(Ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  c = ctx_root(c);
  if (bytes == 0) bytes = 1;
  if (c->budget && c->in_use + bytes > c->budget) {
    set_error("HBM budget exceeded: %zu in use + %zu requested > %zu", c->in_use.load(), bytes, c->budget);
    return ED_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes: out of device memory", bytes);
    return ED_ERR_OOM;
  }
  if (e != cudaSuccess) {
    set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  c->in_use += bytes;
  return ED_OK;
}

void dev_free(Ctx* c, void* p, size_t bytes) {
  if (!p) return;
  c = ctx_root(c);
  cudaFree(p);
  if (bytes == 0) bytes = 1;
  size_t cur = c->in_use.load();
  while (!c->in_use.compare_exchange_weak(cur, cur - std::min(cur, bytes))) {
  }
}

int make_sub_ctx(Ctx* parent, Ctx* sub) {
  Ctx* r = ctx_root(parent);
  sub->root = r;
  sub->device = r->device;
  sub->device_name = r->device_name;
  sub->num_sms = r->num_sms;
  sub->smem_optin = r->smem_optin;
  sub->smem_per_sm = r->smem_per_sm;
  sub->d_binom = r->d_binom;  // read-only, owned by the root
  ED_TRY(dev_alloc_n(sub, &sub->d_red, kRedSlots));
  if (cudaMallocHost(&sub->h_red, 4096) != cudaSuccess) {
    dev_free(sub, sub->d_red, kRedSlots * sizeof(double));
    sub->d_red = nullptr;
    set_error("cudaMallocHost failed");
    return ED_ERR_OOM;
  }
  return ED_OK;
}

void free_sub_ctx(Ctx* sub) {
  dev_free(sub, sub->d_red, kRedSlots * sizeof(double));
  sub->d_red = nullptr;
  if (sub->h_red) cudaFreeHost(sub->h_red);
  sub->h_red = nullptr;
}

int convert_async(const void* src, int sp, void* dst, int dp, uint64_t n, cudaStream_t st);
int lanczos_run(Sector* s, const ed_lanczos_opts* o, double* evals, void* evecs, ed_lanczos_info* info,
                cudaStream_t st);
int trlan_run(Sector* s, const ed_trlan_opts* o, double* evals, void* evecs, ed_trlan_info* info,
              cudaStream_t st);
int autotune(Sector* s, int reps, ed_tune_result* out, cudaStream_t st);
int dmft_update(Ctx* ctx, int n_w, double beta, const double* G_imp, double eps_d, double mu, int n_bath,
                const double* eps_in, const double* V_in, int n_e, const double* e, const double* w, int n_fit,
                double* eps_out, double* V_out, double* chi2, double* sigma, double* G_loc, double* delta_new,
                cudaStream_t st);
int tune_cache_save(Ctx* c, const char* path);
int tune_cache_load(Ctx* c, const char* path, int* n_loaded);
int greens_cf_run(Ctx* ctx, const ed_model* m, int prec, int n_states, const ed_state* states, double beta,
                  int n_w, const double* z, int orbital, int spin, int depth, double boltz_cut, double* G,
                  double* coeffs, cudaStream_t st);

namespace {

__global__ void k_conv(const void* __restrict__ src, int sp, void* __restrict__ dst, int dp, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    double v;
    if (sp == ED_PREC_FP64) v = ((const double*)src)[i];
    else if (sp == ED_PREC_DF64) v = df_to_double(((const float2*)src)[i]);
    else v = (double)((const float*)src)[i];
    if (dp == ED_PREC_FP64) ((double*)dst)[i] = v;
    else if (dp == ED_PREC_DF64) ((float2*)dst)[i] = df_from_double(v);
    else ((float*)dst)[i] = (float)v;
  }
}

__global__ void k_binom(uint32_t* C) {
  int n = threadIdx.x;  // 0..32
  if (n > 32) return;
  for (int k = 0; k <= 32; ++k) {
    uint64_t v = 0;
    if (k <= n) {
      v = 1;
      for (int i = 0; i < k; ++i) v = v * (uint64_t)(n - i) / (uint64_t)(i + 1);
    }
    C[n * 33 + k] = (uint32_t)(v > 0xffffffffull ? 0xffffffffull : v);
  }
}

}  // namespace

int convert_async(const void* src, int sp, void* dst, int dp, uint64_t n, cudaStream_t st) {
  if (!src || !dst) ED_INVALID("NULL vector");
  if (sp < 0 || sp > 2 || dp < 0 || dp > 2) ED_INVALID("unknown precision");
  if (n == 0) return ED_OK;
  uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 152ull * 32);
  k_conv<<<grid, 256, 0, st>>>(src, sp, dst, dp, n);
  ED_LAUNCH_CHECK();
  return ED_OK;
}

}  // namespace ed

using namespace ed;

#define ED_GUARD_BEGIN try {
#define ED_GUARD_END                                   \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    set_error("host allocation failed");               \
    return ED_ERR_OOM;                                 \
  }                                                    \
  catch (...) {                                        \
    set_error("unexpected C++ exception");             \
    return ED_ERR_INVALID;                             \
  }

extern "C" {

int ed_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return ED_ERR_INVALID;
  size_t n = std::min(len - 1, g_err.size());
  std::memcpy(buf, g_err.data(), n);
  buf[n] = 0;
  return ED_OK;
}

int ed_abi_version(void) { return ED_ABI_VERSION; }

int ed_ctx_create(int device, size_t hbm_budget, ed_ctx** out) {
  ED_GUARD_BEGIN
  if (!out) ED_INVALID("out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) {
    set_error("no CUDA device: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) ED_INVALID("device %d outside 0..%d", device, ndev - 1);
  ED_TRY_CUDA(cudaSetDevice(device));
  ed_ctx* h = new ed_ctx();
  Ctx& c = h->c;
  c.device = device;
  c.budget = hbm_budget;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete h;
    set_error("cudaGetDeviceProperties failed");
    return ED_ERR_CUDA;
  }
  if (prop.major < 10) {
    delete h;
    ED_INVALID("device %d is sm_%d%d; this library is built for sm_103a", device, prop.major, prop.minor);
  }
  c.num_sms = prop.multiProcessorCount;
  c.device_name = prop.name;
  c.smem_optin = prop.sharedMemPerBlockOptin;
  c.smem_per_sm = prop.sharedMemPerMultiprocessor;
  int st = dev_alloc_n(&c, &c.d_binom, 33 * 33);
  if (st == ED_OK) st = dev_alloc_n(&c, &c.d_red, kRedSlots);
  if (st == ED_OK && cudaMallocHost(&c.h_red, 4096) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    st = ED_ERR_OOM;
  }
  if (st != ED_OK) {
    ed_ctx_destroy(h);
    return st;
  }
  k_binom<<<1, 33>>>(c.d_binom);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ed_ctx_destroy(h);
    set_error("context set-up kernel failed: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  *out = h;
  return ED_OK;
  ED_GUARD_END
}

int ed_ctx_destroy(ed_ctx* ctx) {
  if (!ctx) return ED_OK;
  Ctx& c = ctx->c;
  cudaSetDevice(c.device);
  dev_free(&c, c.d_binom, 33 * 33 * sizeof(uint32_t));
  dev_free(&c, c.d_red, kRedSlots * sizeof(double));
  if (c.h_red) cudaFreeHost(c.h_red);
  delete ctx;
  return ED_OK;
}

int ed_ctx_bytes_in_use(const ed_ctx* ctx, size_t* out) {
  if (!ctx || !out) ED_INVALID("NULL argument");
  *out = ctx->c.in_use.load();
  return ED_OK;
}

int ed_sector_create(ed_ctx* ctx, const ed_model* model, int n_up, int n_dn, int prec, unsigned flags,
                     ed_sector** out) {
  ED_GUARD_BEGIN
  if (!ctx || !model || !out) ED_INVALID("NULL argument");
  *out = nullptr;
  if (flags & ~(ED_SECTOR_CSR | ED_SECTOR_GENERIC | ED_SECTOR_ACC_DF)) ED_INVALID("unknown flags 0x%x", flags);
  ed_sector* h = new ed_sector();
  int st = build_sector(&ctx->c, model, n_up, n_dn, prec, &h->s);
  h->s.acc_df = (flags & ED_SECTOR_ACC_DF) != 0;
  if (st == ED_OK && !(flags & ED_SECTOR_GENERIC)) st = build_fast(&h->s);
  if (st == ED_OK && (flags & ED_SECTOR_CSR)) st = build_csr(&h->s);
  if (st != ED_OK) {
    free_sector(&h->s);
    delete h;
    return st;
  }
  *out = h;
  return ED_OK;
  ED_GUARD_END
}

int ed_sector_destroy(ed_sector* s) {
  if (!s) return ED_OK;
  cudaSetDevice(s->s.ctx->device);
  host_xfer_free(s->s.ctx, s->xfer);
  free_sector(&s->s);
  delete s;
  return ED_OK;
}

int ed_sector_get_info(const ed_sector* h, ed_sector_info* out) {
  if (!h || !out) ED_INVALID("NULL argument");
  const Sector& s = h->s;
  out->n_s = s.n_s;
  out->n_up = s.n_up;
  out->n_dn = s.n_dn;
  out->prec = s.prec;
  out->D_up = s.up.D;
  out->D_dn = s.dn.D;
  out->dim = s.dim;
  out->hops_up = s.up.n_hops;
  out->hops_dn = s.dn.n_hops;
  out->mix_up = s.n_mix;
  out->csr_nnz = s.csr_nnz;
  out->table_bytes = s.table_bytes;
  // mean entries per row: 1 + mean down hops + mean up hops + mean valid mixed
  double mix = 0.0;
  if (s.n_mix && s.up.D && s.dn.D) {
    // each mixed entry is valid for the fraction of down strings whose move exists:
    // with x occupied and y empty, C(n_s-2, n_dn-1) of C(n_s, n_dn) strings
    double num = 1.0, den = 1.0;
    int nd = s.n_dn, ns = s.n_s;
    if (nd >= 1 && nd <= ns - 1) {
      // C(ns-2, nd-1) / C(ns, nd) = nd (ns - nd) / (ns (ns - 1))
      num = (double)nd * (ns - nd);
      den = (double)ns * (ns - 1);
      mix = (double)s.n_mix / s.up.D * (num / den);
    }
  }
  int fk = 0, fb = 0, fm = 0;
  if (s.fast.ok) fast_variant_info(s.prec, fast_variant_applies(&s, s.tune) ? s.tune : fast_default_variant(&s), &fk, &fb, &fm);
  out->kernel = s.fast.ok ? fk : ((s.dn.D >= 1024 && (size_t)s.dn.D * elem_bytes(s.prec) <= 96 * 1024) ? 1 : 0);
  out->nnz_per_row = 1.0 + (double)s.dn.n_hops / std::max<uint32_t>(s.dn.D, 1) +
                     (double)s.up.n_hops / std::max<uint32_t>(s.up.D, 1) + mix;
  return ED_OK;
}

int ed_sector_basis(const ed_sector* h, int spin, uint32_t* host_out) {
  if (!h || !host_out) ED_INVALID("NULL argument");
  if (spin != ED_SPIN_UP && spin != ED_SPIN_DN) ED_INVALID("spin must be 0 or 1");
  const SpinTables& t = spin == ED_SPIN_UP ? h->s.up : h->s.dn;
  ED_TRY_CUDA(cudaSetDevice(h->s.ctx->device));
  ED_TRY_CUDA(cudaMemcpy(host_out, t.basis, sizeof(uint32_t) * t.D, cudaMemcpyDeviceToHost));
  return ED_OK;
}

int ed_sector_hops(const ed_sector* h, int spin, uint32_t* ptr, uint32_t* tgt, double* val) {
  if (!h) ED_INVALID("NULL sector");
  if (spin != ED_SPIN_UP && spin != ED_SPIN_DN) ED_INVALID("spin must be 0 or 1");
  const SpinTables& t = spin == ED_SPIN_UP ? h->s.up : h->s.dn;
  ED_TRY_CUDA(cudaSetDevice(h->s.ctx->device));
  if (ptr) ED_TRY_CUDA(cudaMemcpy(ptr, t.hop_ptr, sizeof(uint32_t) * (t.D + 1), cudaMemcpyDeviceToHost));
  if (t.n_hops) {
    if (tgt) ED_TRY_CUDA(cudaMemcpy(tgt, t.hop_tgt, sizeof(uint32_t) * t.n_hops, cudaMemcpyDeviceToHost));
    if (val) ED_TRY_CUDA(cudaMemcpy(val, t.hop_val, sizeof(double) * t.n_hops, cudaMemcpyDeviceToHost));
  }
  return ED_OK;
}

int ed_sector_csr_rows(const ed_sector* h, uint64_t row0, uint64_t nrows, uint64_t* row_ptr, uint32_t* cols,
                       double* vals) {
  ED_GUARD_BEGIN
  if (!h || !row_ptr) ED_INVALID("NULL argument");
  const Sector& s = h->s;
  if (!s.csr_ptr) ED_INVALID("sector has no stored CSR");
  if (row0 > s.dim || nrows > s.dim - row0) ED_INVALID("row range outside the sector");
  ED_TRY_CUDA(cudaSetDevice(s.ctx->device));
  ED_TRY_CUDA(cudaMemcpy(row_ptr, s.csr_ptr + row0, sizeof(uint64_t) * (nrows + 1), cudaMemcpyDeviceToHost));
  uint64_t base = row_ptr[0], cnt = row_ptr[nrows] - base;
  for (uint64_t i = 0; i <= nrows; ++i) row_ptr[i] -= base;
  if (cnt) {
    if (cols) ED_TRY_CUDA(cudaMemcpy(cols, s.csr_col + base, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost));
    if (vals) ED_TRY_CUDA(cudaMemcpy(vals, s.csr_val + base, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  }
  return ED_OK;
  ED_GUARD_END
}

int ed_apply_h(ed_sector* h, const void* x, void* y, void* stream) {
  if (!h) ED_INVALID("NULL sector");
  return apply_h(&h->s, x, y, as_stream(stream));
}

int ed_apply_h_host(ed_sector* h, uint64_t n_vec, const void* x_host, void* y_host, void* stream) {
  if (!h) ED_INVALID("NULL sector");
  return apply_h_host(&h->s, &h->xfer, n_vec, x_host, y_host, as_stream(stream));
}

int ed_apply_h_csr(ed_sector* h, const void* x, void* y, void* stream) {
  if (!h) ED_INVALID("NULL sector");
  return apply_h_csr(&h->s, x, y, as_stream(stream));
}

int ed_convert(const void* src, int src_prec, void* dst, int dst_prec, uint64_t n, void* stream) {
  return convert_async(src, src_prec, dst, dst_prec, n, as_stream(stream));
}

int ed_dot(ed_ctx* ctx, const void* x, const void* y, uint64_t n, int prec, double* result, void* stream) {
  if (!ctx || !x || !y || !result) ED_INVALID("NULL argument");
  if (n == 0) {
    *result = 0.0;
    return ED_OK;
  }
  cudaStream_t st = as_stream(stream);
  double* d_out = ctx->c.d_red + kRedSlots - 8;
  // partials use the front of the scratch; the result slot sits at its end
  ED_TRY(dot_async(&ctx->c, x, y, n, prec, d_out, st));
  ED_TRY_CUDA(cudaMemcpyAsync(ctx->c.h_red, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  *result = ctx->c.h_red[0];
  return ED_OK;
}

int ed_lanczos(ed_sector* h, const ed_lanczos_opts* opts, double* evals, void* evecs, ed_lanczos_info* info,
               void* stream) {
  ED_GUARD_BEGIN
  if (!h || !opts || !evals) ED_INVALID("NULL argument");
  if (opts->k < 1 || opts->k > ED_MAX_K) ED_INVALID("k=%d outside 1..%d", opts->k, ED_MAX_K);
  if (opts->max_iter < 1) ED_INVALID("max_iter must be >= 1");
  if (!(opts->tol > 0.0)) ED_INVALID("tol must be positive");
  if (info) std::memset(info, 0, sizeof(*info));
  ED_TRY_CUDA(cudaSetDevice(h->s.ctx->device));
  return lanczos_run(&h->s, opts, evals, evecs, info, as_stream(stream));
  ED_GUARD_END
}

int ed_dmft_update(ed_ctx* ctx, int n_w, double beta, const double* G_imp, double eps_d, double mu, int n_bath,
                   const double* eps_in, const double* V_in, int n_e, const double* e, const double* w, int n_fit,
                   double* eps_out, double* V_out, double* chi2, double* sigma, double* G_loc, double* delta_new,
                   void* stream) {
  ED_GUARD_BEGIN
  if (!ctx) ED_INVALID("NULL argument");
  ED_TRY_CUDA(cudaSetDevice(ctx->c.device));
  return dmft_update(&ctx->c, n_w, beta, G_imp, eps_d, mu, n_bath, eps_in, V_in, n_e, e, w, n_fit, eps_out, V_out,
                     chi2, sigma, G_loc, delta_new, as_stream(stream));
  ED_GUARD_END
}

int ed_sector_autotune(ed_sector* h, int reps, ed_tune_result* out, void* stream) {
  ED_GUARD_BEGIN
  if (!h || !out) ED_INVALID("NULL argument");
  ED_TRY_CUDA(cudaSetDevice(h->s.ctx->device));
  return autotune(&h->s, reps, out, as_stream(stream));
  ED_GUARD_END
}

int ed_sector_set_variant(ed_sector* h, int variant) {
  ED_GUARD_BEGIN
  if (!h) ED_INVALID("NULL argument");
  if (variant != -1 && !fast_variant_applies(&h->s, variant))
    ED_INVALID("H*v variant %d does not apply to this sector", variant);
  h->s.tune = variant;
  return ED_OK;
  ED_GUARD_END
}

int ed_sector_get_variant(const ed_sector* h, int* variant) {
  ED_GUARD_BEGIN
  if (!h || !variant) ED_INVALID("NULL argument");
  *variant = fast_variant_applies(&h->s, h->s.tune) ? h->s.tune : -1;
  return ED_OK;
  ED_GUARD_END
}

int ed_tune_cache_save(ed_ctx* ctx, const char* path) {
  ED_GUARD_BEGIN
  if (!ctx || !path) ED_INVALID("NULL argument");
  return tune_cache_save(&ctx->c, path);
  ED_GUARD_END
}

int ed_tune_cache_load(ed_ctx* ctx, const char* path, int* n_loaded) {
  ED_GUARD_BEGIN
  if (!ctx || !path) ED_INVALID("NULL argument");
  int n = 0;
  const int st = tune_cache_load(&ctx->c, path, &n);
  if (n_loaded) *n_loaded = n;
  return st;
  ED_GUARD_END
}

int ed_lanczos_tr(ed_sector* h, const ed_trlan_opts* opts, double* evals, void* evecs, ed_trlan_info* info,
                  void* stream) {
  ED_GUARD_BEGIN
  if (!h || !opts || !evals) ED_INVALID("NULL argument");
  if (opts->max_iter < 1) ED_INVALID("max_iter must be >= 1");
  if (info) std::memset(info, 0, sizeof(*info));
  ED_TRY_CUDA(cudaSetDevice(h->s.ctx->device));
  return trlan_run(&h->s, opts, evals, evecs, info, as_stream(stream));
  ED_GUARD_END
}

int ed_greens_cf(ed_ctx* ctx, const ed_model* model, int prec, int n_states, const ed_state* states, double beta,
                 int n_w, int orbital, int spin, int depth, double boltz_cut, double* G, double* coeffs,
                 void* stream) {
  ED_GUARD_BEGIN
  if (!ctx || !model) ED_INVALID("NULL argument");
  ED_TRY_CUDA(cudaSetDevice(ctx->c.device));
  return greens_cf_run(&ctx->c, model, prec, n_states, states, beta, n_w, nullptr, orbital, spin, depth,
                       boltz_cut, G, coeffs, as_stream(stream));
  ED_GUARD_END
}

int ed_greens_cf_z(ed_ctx* ctx, const ed_model* model, int prec, int n_states, const ed_state* states,
                   double beta, int n_z, const double* z, int orbital, int spin, int depth, double boltz_cut,
                   double* G, double* coeffs, void* stream) {
  ED_GUARD_BEGIN
  if (!ctx || !model || !z) ED_INVALID("NULL argument");
  ED_TRY_CUDA(cudaSetDevice(ctx->c.device));
  return greens_cf_run(&ctx->c, model, prec, n_states, states, beta, n_z, z, orbital, spin, depth, boltz_cut, G,
                       coeffs, as_stream(stream));
  ED_GUARD_END
}

}  // extern "C"
