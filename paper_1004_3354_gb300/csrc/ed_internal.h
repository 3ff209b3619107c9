// Internal declarations of libedgb: device table layout, arithmetic policies,
// allocation and error helpers.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/ed.h"

namespace ed {

// ------------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

#define ED_TRY_CUDA(call)                                                          \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::ed::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e),      \
                      __FILE__, __LINE__);                                         \
      return ED_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

#define ED_TRY(call)                 \
  do {                               \
    int _s = (call);                 \
    if (_s != ED_OK) return _s;      \
  } while (0)

#define ED_INVALID(...)              \
  do {                               \
    ::ed::set_error(__VA_ARGS__);    \
    return ED_ERR_INVALID;           \
  } while (0)

// Launch-error check after a kernel launch (asynchronous errors surface later).
#define ED_LAUNCH_CHECK() ED_TRY_CUDA(cudaGetLastError())

// ------------------------------------------------------------------ context
struct Ctx {
  int device = 0;
  std::string device_name;       // cudaDeviceProp::name, keys the autotune cache
  std::mutex tune_mu;
  std::map<std::string, int> tune_cache;  // sector shape key -> fast H*v variant
  size_t budget = 0;      // 0 = unlimited
  std::atomic<size_t> in_use{0};
  int num_sms = 0;
  size_t smem_optin = 0;
  size_t smem_per_sm = 0;        // shared memory of one SM (all resident blocks)
  uint32_t* d_binom = nullptr;   // [33][33] binomial coefficients C(n, k)
  double* d_red = nullptr;       // reduction scratch (partials), kRedSlots doubles
  double* h_red = nullptr;       // pinned host mirror of d_red[0..63]
  // A sub-context (a worker thread of the request server) has its own
  // reduction scratch and charges its allocations to, and shares the autotune
  // cache of, the context it was made from.
  Ctx* root = nullptr;
};

inline Ctx* ctx_root(Ctx* c) { return c->root ? c->root : c; }
// Make sub a sub-context of parent (own reduction scratch, parent's budget,
// device tables and autotune cache); free_sub_ctx releases its scratch.
int make_sub_ctx(Ctx* parent, Ctx* sub);
void free_sub_ctx(Ctx* sub);

constexpr int kRedSlots = 8192;

int dev_alloc(Ctx* c, void** p, size_t bytes);
void dev_free(Ctx* c, void* p, size_t bytes);

template <class T>
int dev_alloc_n(Ctx* c, T** p, size_t n) {
  return dev_alloc(c, reinterpret_cast<void**>(p), n * sizeof(T));
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Raise a kernel's dynamic shared-memory cap to the device's opt-in maximum
// before a launch that needs `need` bytes.  Every call sets the same value, so
// host threads that launch one kernel with different sizes (server workers,
// sectors of several sizes) cannot undo each other's setting between set and
// launch; occupancy still follows each launch's own size.
template <class K>
int smem_cap(const Ctx* c, K kern, size_t need) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) {
    set_error("cudaFuncGetAttributes failed: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  const size_t cap = c->smem_optin > fa.sharedSizeBytes ? c->smem_optin - fa.sharedSizeBytes : 0;  // per kernel
  if (need > cap) {
    set_error("kernel needs %zu bytes of dynamic shared memory, more than the %zu a block may have", need, cap);
    return ED_ERR_INVALID;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  if (e != cudaSuccess) {
    set_error("cudaFuncSetAttribute failed: %s", cudaGetErrorString(e));
    return ED_ERR_CUDA;
  }
  return ED_OK;
}

// The context behind an opaque handle (abi.cu).
Ctx* ctx_of(ed_ctx* h);

// --------------------------------------------------------- sector on device
// Per-spin tables (device pointers).  Strings are uint32 bit masks.
struct SpinTables {
  int n = 0;                 // particles of this spin
  uint32_t D = 0;            // number of strings C(n_s, n)
  uint64_t n_hops = 0;
  uint32_t* basis = nullptr;     // [D] ascending
  uint32_t* hop_ptr = nullptr;   // [D+1]
  uint32_t* hop_tgt = nullptr;   // [n_hops] rank of the string reached
  double* hop_val = nullptr;     // [n_hops] T_ij * sign
  float2* hop_val_df = nullptr;  // [n_hops] same value split hi + lo
  double* e = nullptr;           // [D] one-spin diagonal part
  float2* e_df = nullptr;
  uint32_t max_hops = 0;         // longest hop list
};

// Kernel-side view of a sector, passed by value.
struct SectorView {
  uint32_t D_up, D_dn;
  int n_s, M;
  // cross (up x down) diagonal tables over the K sites w_lo .. w_lo + K - 1,
  // split into chunks of at most 8 sites: u_c = (u >> (w_lo + 8c)) & mask_c,
  // W_c[u_c][d_c] at w_off[c] + (u_c << w_bits[c]) + d_c
  int w_lo;
  int n_chunks;
  int w_bits[4];
  uint32_t w_off[4];
  const double* W;
  const float2* W_df;
  // one-body gather lists
  const uint32_t *uh_ptr, *uh_tgt, *dh_ptr, *dh_tgt;
  const double *uh_val, *dh_val;
  const float2 *uh_val_df, *dh_val_df;
  const double *e_up, *e_dn;
  const float2 *e_up_df, *e_dn_df;
  // spin-flip / pair-hop: per up string a list of (u_c, J * s_u, down-move table)
  const uint32_t *mx_ptr, *mx_tgt;
  const double* mx_val;
  const float2* mx_val_df;
  const uint8_t* mx_mv;
  // down-move tables [M*M][D_dn]: (rank << 1 | sign bit) or -1
  const int32_t* dn_move;
};

struct Sector {
  Ctx* ctx = nullptr;
  int n_s = 0, n_up = 0, n_dn = 0, prec = 0, M = 0, K = 0, orb0 = 0, w_lo = 0;
  double T[ED_MAX_SITES * ED_MAX_SITES];
  double U_site[ED_MAX_SITES];
  double Up = 0, J = 0, Jsf = 0, Jph = 0;
  SpinTables up, dn;
  uint64_t dim = 0;
  // cross tables
  int n_chunks = 0;
  int w_bits[4] = {0, 0, 0, 0};
  uint32_t w_off[4] = {0, 0, 0, 0};
  uint32_t w_size = 0;
  double* W = nullptr;
  float2* W_df = nullptr;
  // mixed terms
  uint64_t n_mix = 0;
  uint32_t max_mix = 0;
  uint32_t *mx_ptr = nullptr, *mx_tgt = nullptr;
  double* mx_val = nullptr;
  float2* mx_val_df = nullptr;
  uint8_t* mx_mv = nullptr;
  int32_t* dn_move = nullptr;
  // tables of the fast row kernel (apply_fast.cu); fast.ok = false -> generic kernels
  struct Fast {
    // Window layout: the down strings are cut into windows of 128 consecutive
    // ranks; inside a window they are sorted by hop count (longest first) and
    // dealt to 32 lanes x 4 slots, entry index w*128 + lane*4 + slot.
    bool ok = false;
    uint32_t n_win = 0;         // ceil(D_dn / 128)
    uint32_t max_cnt = 0;       // widest down-hop list
    int n_coef = 0;             // distinct down-hop matrix elements (<= 256), one of them 0.0
    int n_pat = 1;              // 2^K diagonal patterns of the up string
    uint32_t* perm = nullptr;   // [n_win*128] down rank of each entry (D_dn for padding)
    uint8_t* cnt = nullptr;     // [n_win*4] longest list in each slot
    uint32_t* hop = nullptr;    // [n_win][max_cnt][32][4] (x byte offset << 13) | coefficient byte offset
    double* coef = nullptr;     // [n_coef]
    float2* coef_df = nullptr;
    double* dd = nullptr;       // [n_pat][n_win*128] e_dn[d] + W[p_u][pattern(d)]
    float2* dd_df = nullptr;
    uint32_t* row_order = nullptr;  // [D_up] rows grouped by one-body connected component
    uint32_t* row_pat = nullptr;    // [D_up] diagonal pattern of each up string
    // orbitals on the top sites: down strings come in blocks of equal impurity
    // pattern, and an impurity move shifts a rank by a per-pattern constant
    bool mix_delta = false;
    uint8_t* dpat = nullptr;        // [n_win*128] impurity pattern of each entry
    uint32_t* wpat = nullptr;       // [n_win] pattern shared by a whole window, or ~0u
    int32_t* mdelta = nullptr;      // [M*M][2^M] (shift << 1 | sign) or INT32_MIN
    int n_lp = 1;                   // term lists per row in the row kernel (2^M with mix_delta)
    uint32_t lcap = 1;              // entries of one list: longest up-hop + spin-flip/pair-hop list
    // two-row kernel (double-float and float vectors): rows are processed in
    // pairs (row_order[2i], row_order[2i+1]) staged interleaved; its hop words
    // hold byte offsets into that interleaved row and into a table of 16-byte
    // coefficient entries
    bool pair_ok = false;
    uint32_t* hop2 = nullptr;   // [n_win][max_cnt][32][4] two-row encoding
    // natural-order kernel for float vectors (apply_nat.cu): lane l of a warp
    // owns down string 32 g + l, R up strings per block
    bool nat_ok = false;
    uint32_t nat_grp = 0;           // ceil(D_dn / 32)
    uint32_t nat_mc = 0;            // hop slots per string: max_cnt rounded up to even
    uint32_t* nat_hop = nullptr;    // [nat_grp][nat_mc/2][32][2]: target rank << 8 | coefficient id
    uint32_t* nat_meta = nullptr;   // [nat_grp*32]: hop count | diagonal pattern << 8 | impurity pattern << 16
    float* nat_edn = nullptr;       // [nat_grp*32] e_dn as float
    float* nat_coef = nullptr;      // [n_coef] down-hop coefficients as float
    float* nat_W = nullptr;         // [n_pat][n_pat] cross diagonal table as float
    float2* nat_dd = nullptr;       // [n_pat][nat_grp*32] double-float e_dn[d] + W[pu][pattern(d)] (DF64)
  } fast;
  // autotuned H*v variant of the fast path (apply_fast.cu), -1 = untuned
  int tune = -1;
  // FP32 vectors with double-float sums (ED_SECTOR_ACC_DF): no natural-order tables
  bool acc_df = false;
  // stored CSR (optional)
  uint64_t csr_nnz = 0;
  uint64_t* csr_ptr = nullptr;
  uint32_t* csr_col = nullptr;
  double* csr_val = nullptr;
  // bookkeeping of allocations: (pointer, bytes)
  std::vector<std::pair<void*, size_t>> allocs;
  size_t table_bytes = 0;

  SectorView view() const;
};

template <class T>
int sector_alloc(Sector* s, T** p, size_t n) {
  if (n == 0) n = 1;
  int st = dev_alloc(s->ctx, reinterpret_cast<void**>(p), n * sizeof(T));
  if (st == ED_OK) {
    s->allocs.push_back({(void*)*p, n * sizeof(T)});
    s->table_bytes += n * sizeof(T);
  }
  return st;
}

// Builders (basis.cu, csr.cu)
int validate_model(const ed_model* m);
int build_sector(Ctx* ctx, const ed_model* m, int n_up, int n_dn, int prec, Sector* s);
int build_csr(Sector* s);
void free_sector(Sector* s);

// Fast row kernel set-up (apply_fast.cu); leaves fast.ok false when unsupported.
int build_fast(Sector* s);
// With dotp != NULL the kernel also writes per-block partial sums of <x, Hx>
// to dotp[0 .. *nparts).
int apply_fast(const Sector* s, const void* x, void* y, cudaStream_t st, double* dotp = nullptr,
               int* nparts = nullptr);
// Autotune cache key of a sector's shape (tune.cu); the cached variant is
// applied when a sector with that key is created.
std::string tune_key(const Sector* s);
void tune_apply_cached(Sector* s);

// Natural-order kernel for float and double-float sectors (apply_nat.cu):
// tables, launch of variant v in [0, kNatVariants), its rows per block /
// launch shape (they depend on the sector's format) and shared memory.
constexpr int kNatVariants = 6;
int build_nat(Sector* s, const std::vector<double>& coef, int zero_id);
int launch_nat(const Sector* s, int v, const void* x, void* y, cudaStream_t st, double* dotp, int* nparts);
void nat_variant_info(int prec, int v, int* rows, int* block, int* min_blocks);
size_t nat_variant_smem(const Sector* s, int v);

// Variants of the fast H*v path (apply_fast.cu): index v in [0, fast_variants()).
int fast_variants();
void fast_variant_info(int prec, int v, int* kernel, int* block, int* min_blocks);
bool fast_variant_applies(const Sector* s, int v);
int fast_default_variant(const Sector* s);
int apply_fast_variant(const Sector* s, int v, const void* x, void* y, cudaStream_t st, double* dotp = nullptr,
                       int* nparts = nullptr);

// Host-buffer H*v (hostio.cu): pipelined copies and applies over n_vec vectors;
// the device buffers and streams are made at the first call and kept in *hp.
struct HostXfer;
int apply_h_host(Sector* s, HostXfer** hp, uint64_t n_vec, const void* xh, void* yh, cudaStream_t st);
void host_xfer_free(Ctx* c, HostXfer* h);

// Apply entry points (apply.cu, csr.cu)
int apply_h(const Sector* s, const void* x, void* y, cudaStream_t st);
int apply_h_csr(const Sector* s, const void* x, void* y, cudaStream_t st);

// Vector helpers (lanczos.cu)
size_t elem_bytes(int prec);
int dot_async(Ctx* c, const void* x, const void* y, uint64_t n, int prec, double* d_out,
              cudaStream_t st);
int convert_async(const void* src, int sp, void* dst, int dp, uint64_t n, cudaStream_t st);

// Sector-change maps for c+ / c (basis.cu): phi = op psi, target sector t from s.
int apply_cop(const Sector* src, const Sector* dst, int orbital, int spin, bool dagger,
              const void* psi, void* phi, cudaStream_t st);

// Lanczos coefficient recurrence without reorthogonalisation (lanczos.cu),
// used by the Green's function: returns n2 = <phi|phi>, a[0..L), b[0..L) (b[0]=0).
int lanczos_coeffs(Sector* s, const void* phi, int depth, double* n2, double* a, double* b,
                   int* L, cudaStream_t st);

// ------------------------------------------------------ double-float maths
// Error-free transformations (Knuth's TwoSum, Dekker/Kahan TwoProduct via FMA).
// The explicit _rn intrinsics keep the compiler from contracting a product
// into a following sum, which would break the error-free property.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// acc (hi, lo) += c (hi, lo) * x (hi, lo); the lo part accumulates lazily.
__device__ __forceinline__ void df_mac(float2& acc, float2 c, float2 x) {
  float p = __fmul_rn(c.x, x.x);
  float e = __fmaf_rn(c.x, x.x, -p);
  e = __fmaf_rn(c.x, x.y, e);
  e = __fmaf_rn(c.y, x.x, e);
  float s, t;
  two_sum(acc.x, p, s, t);
  acc.x = s;
  acc.y = __fadd_rn(acc.y, __fadd_rn(t, e));
}

// acc += c * x with x a plain float.
__device__ __forceinline__ void df_mac1(float2& acc, float2 c, float x) {
  float p = __fmul_rn(c.x, x);
  float e = __fmaf_rn(c.x, x, -p);
  e = __fmaf_rn(c.y, x, e);
  float s, t;
  two_sum(acc.x, p, s, t);
  acc.x = s;
  acc.y = __fadd_rn(acc.y, __fadd_rn(t, e));
}

// Two independent double-float accumulators at once with the paired FP32
// instructions (add/sub/mul/fma .f32x2): H = (hi0, hi1), L = (lo0, lo1) take
// (Ch, Cl) * (Xh, Xl) lane-wise, each lane exactly as df_mac (or as df_mac1
// when XLO is false and x is a plain float).
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

template <bool XLO>
__device__ __forceinline__ void df_mac2(float2& H, float2& L, float2 Ch, float2 Cl, float2 Xh, float2 Xl) {
  const float2 P = __fmul2_rn(Ch, Xh);
  float2 E = __ffma2_rn(Ch, Xh, make_float2(-P.x, -P.y));
  if (XLO) E = __ffma2_rn(Ch, Xl, E);
  E = __ffma2_rn(Cl, Xh, E);
  const float2 S = __fadd2_rn(H, P);
  const float2 BB = f2_sub(S, H);
  const float2 T = __fadd2_rn(f2_sub(H, f2_sub(S, BB)), f2_sub(P, BB));
  H = S;
  L = __fadd2_rn(L, __fadd2_rn(T, E));
}

__device__ __forceinline__ float2 df_norm(float2 a) {
  float s, e;
  fast_two_sum(a.x, a.y, s, e);
  return make_float2(s, e);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  return df_norm(make_float2(s, e));
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// double <-> double-float (set-up and boundary conversions only).
__host__ __device__ inline float2 df_from_double(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  return make_float2(hi, lo);
}
__host__ __device__ inline double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// ------------------------------------------------------ arithmetic policies
// A policy fixes the stored element type V, the accumulator A, the matrix
// coefficient type C (read from the double or the double-float copy of a
// table) and how one coefficient multiplies one element.
struct PolF64 {
  using V = double;
  using A = double;
  using C = double;
  static constexpr int prec = ED_PREC_FP64;
  __device__ static __forceinline__ A zero() { return 0.0; }
  __device__ static __forceinline__ C ld(const double* d, const float2*, size_t k) { return d[k]; }
  __device__ static __forceinline__ const C* ld_ptr(const double* d, const float2*) { return d; }
  __device__ static __forceinline__ C neg(C c) { return -c; }
  __device__ static __forceinline__ void mac(A& a, C c, V x) { a = fma(c, x, a); }
  __device__ static __forceinline__ V out(A a) { return a; }
  __device__ static __forceinline__ void dot(A& a, V x, V y) { a = fma(x, y, a); }
  __device__ static __forceinline__ A warp_sum(A a) {
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  }
  __device__ static __forceinline__ double to_double(A a) { return a; }
};

struct PolDF {
  using V = float2;
  using A = float2;
  using C = float2;
  static constexpr int prec = ED_PREC_DF64;
  __device__ static __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ C ld(const double*, const float2* f, size_t k) { return f[k]; }
  __device__ static __forceinline__ const C* ld_ptr(const double*, const float2* f) { return f; }
  __device__ static __forceinline__ C neg(C c) { return make_float2(-c.x, -c.y); }
  __device__ static __forceinline__ void mac(A& a, C c, V x) { df_mac(a, c, x); }
  __device__ static __forceinline__ V out(A a) { return df_norm(a); }
  __device__ static __forceinline__ void dot(A& a, V x, V y) { df_mac(a, x, y); }
  __device__ static __forceinline__ A warp_sum(A a) {
    for (int o = 16; o > 0; o >>= 1)
      a = df_add(a, make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)));
    return a;
  }
  __device__ static __forceinline__ double to_double(A a) { return (double)a.x + (double)a.y; }
};

struct PolF32 {
  using V = float;
  using A = float2;
  using C = float2;
  static constexpr int prec = ED_PREC_FP32;
  __device__ static __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ C ld(const double*, const float2* f, size_t k) { return f[k]; }
  __device__ static __forceinline__ const C* ld_ptr(const double*, const float2* f) { return f; }
  __device__ static __forceinline__ C neg(C c) { return make_float2(-c.x, -c.y); }
  __device__ static __forceinline__ void mac(A& a, C c, V x) { df_mac1(a, c, x); }
  __device__ static __forceinline__ V out(A a) { return __fadd_rn(a.x, a.y); }
  __device__ static __forceinline__ void dot(A& a, V x, V y) { df_mac1(a, make_float2(x, 0.f), y); }
  __device__ static __forceinline__ A warp_sum(A a) {
    for (int o = 16; o > 0; o >>= 1)
      a = df_add(a, make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)));
    return a;
  }
  __device__ static __forceinline__ double to_double(A a) { return (double)a.x + (double)a.y; }
};

}  // namespace ed
