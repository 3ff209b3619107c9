// Autotuner of the fast H*v path: per sector, time every applicable variant
// (one or two up strings per block, times the launch shapes of apply_fast.cu)
// on the device and keep the fastest.  Results are cached in the context under
// a key of the sector's shape and can be saved to / loaded from a JSON file
// (entries measured on another GPU model are ignored when loading).
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ed_internal.h"

namespace ed {

namespace {

__global__ void k_tune_fill(uint32_t* __restrict__ p, uint64_t words, uint64_t seed, int prec) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x) {
    // splitmix64 of the index: uniform values in [-1, 1) of the element type
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    if (prec == ED_PREC_FP64) {
      reinterpret_cast<double*>(p)[i] = u;
    } else if (prec == ED_PREC_DF64) {
      reinterpret_cast<float2*>(p)[i] = make_float2((float)u, 0.f);
    } else {
      reinterpret_cast<float*>(p)[i] = (float)u;
    }
  }
}

}  // namespace

std::string tune_key(const Sector* s) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "prec=%d n_s=%d M=%d orb0=%d D_up=%u D_dn=%u up_hops=%u dn_hops=%u mix=%llu",
                s->prec, s->n_s, s->M, s->orb0, s->up.D, s->dn.D, s->up.max_hops, s->dn.max_hops,
                (unsigned long long)s->n_mix);
  return buf;
}

void tune_apply_cached(Sector* s) {
  if (!s->fast.ok) return;
  Ctx* c = s->ctx;
  c = ctx_root(c);
  std::lock_guard<std::mutex> lk(c->tune_mu);
  auto it = c->tune_cache.find(tune_key(s));
  if (it != c->tune_cache.end() && fast_variant_applies(s, it->second)) s->tune = it->second;
}

int autotune(Sector* s, int reps, ed_tune_result* out, cudaStream_t st) {
  std::memset(out, 0, sizeof(*out));
  out->chosen = -1;
  if (!s->fast.ok) return ED_OK;  // only the generic kernels: nothing to choose
  reps = std::max(1, std::min(reps, 50));
  const size_t eb = elem_bytes(s->prec);
  void *x = nullptr, *y = nullptr;
  ED_TRY(dev_alloc(s->ctx, &x, s->dim * eb));
  struct Free {
    Ctx* c;
    void* p;
    size_t b;
    ~Free() {
      if (p) dev_free(c, p, b);
    }
  } fx{s->ctx, x, s->dim * eb};
  ED_TRY(dev_alloc(s->ctx, &y, s->dim * eb));
  Free fy{s->ctx, y, s->dim * eb};
  const uint64_t words = s->dim;
  k_tune_fill<<<(unsigned)std::min<uint64_t>((words + 255) / 256, 4096), 256, 0, st>>>(
      static_cast<uint32_t*>(x), words, 0x5eedull, s->prec);
  ED_LAUNCH_CHECK();
  cudaEvent_t a, b;
  ED_TRY_CUDA(cudaEventCreate(&a));
  ED_TRY_CUDA(cudaEventCreate(&b));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{a, b};
  const int nv = std::min(fast_variants(), ED_MAX_TUNE);
  double best = 0.0;
  for (int v = 0; v < nv; ++v) {
    const int i = out->n_candidates++;
    fast_variant_info(s->prec, v, &out->kernel[i], &out->block[i], &out->min_blocks[i]);
    out->ms[i] = -1.0;
    if (!fast_variant_applies(s, v)) continue;
    // a launch shape that does not fit the SM is reported and skipped
    if (apply_fast_variant(s, v, x, y, st) != ED_OK) continue;
    ED_TRY(apply_fast_variant(s, v, x, y, st));
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) {
      ED_TRY_CUDA(cudaEventRecord(a, st));
      ED_TRY(apply_fast_variant(s, v, x, y, st));
      ED_TRY_CUDA(cudaEventRecord(b, st));
      ED_TRY_CUDA(cudaEventSynchronize(b));
      ED_TRY_CUDA(cudaEventElapsedTime(&t[r], a, b));
    }
    std::sort(t.begin(), t.end());
    out->ms[i] = t[reps / 2];
    if (out->chosen < 0 || out->ms[i] < best) {
      best = out->ms[i];
      out->chosen = i;
    }
  }
  set_error("");
  if (out->chosen >= 0) {
    s->tune = out->chosen;  // candidate i is variant i
    Ctx* r = ctx_root(s->ctx);
    std::lock_guard<std::mutex> lk(r->tune_mu);
    r->tune_cache[tune_key(s)] = s->tune;
  }
  return ED_OK;
}

// ------------------------------------------------------------------ JSON
static std::string json_escape(const std::string& v) {
  std::string o;
  for (char ch : v) {
    if (ch == '"' || ch == '\\') o += '\\';
    o += ch;
  }
  return o;
}

int tune_cache_save(Ctx* c, const char* path) {
  std::lock_guard<std::mutex> lk(c->tune_mu);
  std::ofstream f(path);
  if (!f) ED_INVALID("cannot write %s", path);
  f << "{\"format\": \"libedgb-autotune-1\", \"device\": \"" << json_escape(c->device_name) << "\", \"entries\": [";
  bool first = true;
  for (const auto& kv : c->tune_cache) {
    int k = 0, bs = 0, mb = 0, prec = 0;
    std::sscanf(kv.first.c_str(), "prec=%d", &prec);  // the key starts with the sector's format
    fast_variant_info(prec, kv.second, &k, &bs, &mb);
    f << (first ? "\n" : ",\n") << "  {\"key\": \"" << json_escape(kv.first) << "\", \"variant\": " << kv.second
      << ", \"kernel\": " << k << ", \"block\": " << bs << ", \"min_blocks\": " << mb << "}";
    first = false;
  }
  f << "\n]}\n";
  if (!f) ED_INVALID("write to %s failed", path);
  return ED_OK;
}

namespace {

// Tokens of a JSON text: strings (unescaped) and bare words (numbers, true,
// false, null) in order, punctuation dropped.  Enough for the flat file
// tune_cache_save writes; anything else is rejected by the caller.
bool json_tokens(const std::string& t, std::vector<std::pair<bool, std::string>>& out) {
  size_t i = 0;
  while (i < t.size()) {
    const char ch = t[i];
    if (ch == '"') {
      std::string v;
      ++i;
      while (i < t.size() && t[i] != '"') {
        if (t[i] == '\\' && i + 1 < t.size()) ++i;
        v += t[i++];
      }
      if (i >= t.size()) return false;
      ++i;
      out.emplace_back(true, v);
    } else if (std::isalnum((unsigned char)ch) || ch == '-' || ch == '+' || ch == '.') {
      std::string v;
      while (i < t.size() && (std::isalnum((unsigned char)t[i]) || t[i] == '-' || t[i] == '+' || t[i] == '.'))
        v += t[i++];
      out.emplace_back(false, v);
    } else {
      ++i;
    }
  }
  return true;
}

}  // namespace

int tune_cache_load(Ctx* c, const char* path, int* n_loaded) {
  std::ifstream f(path);
  if (!f) ED_INVALID("cannot read %s", path);
  std::stringstream ss;
  ss << f.rdbuf();
  std::vector<std::pair<bool, std::string>> tk;
  if (!json_tokens(ss.str(), tk)) ED_INVALID("%s: unterminated string", path);
  auto value_of = [&](size_t from, const char* name, size_t* at) -> const std::string* {
    for (size_t i = from; i + 1 < tk.size(); ++i)
      if (tk[i].first && tk[i].second == name) {
        *at = i + 1;
        return &tk[i + 1].second;
      }
    return nullptr;
  };
  size_t at = 0;
  const std::string* fmt = value_of(0, "format", &at);
  if (!fmt || *fmt != "libedgb-autotune-1") ED_INVALID("%s is not a libedgb autotune cache", path);
  const std::string* dev = value_of(0, "device", &at);
  if (!dev) ED_INVALID("%s has no device name", path);
  *n_loaded = 0;
  if (*dev != c->device_name) return ED_OK;  // measured on another GPU model
  std::map<std::string, int> got;
  size_t pos = at;
  while (true) {
    size_t a1 = 0, a2 = 0;
    const std::string* key = value_of(pos, "key", &a1);
    if (!key) break;
    const std::string* var = value_of(a1, "variant", &a2);
    if (!var) ED_INVALID("%s: entry without a variant", path);
    char* end = nullptr;
    const long v = std::strtol(var->c_str(), &end, 10);
    if (end == var->c_str() || *end != '\0' || v < 0 || v >= fast_variants())
      ED_INVALID("%s: bad variant '%s'", path, var->c_str());
    got[*key] = (int)v;
    pos = a2;
  }
  std::lock_guard<std::mutex> lk(c->tune_mu);
  for (const auto& kv : got) c->tune_cache[kv.first] = kv.second;
  *n_loaded = (int)got.size();
  return ED_OK;
}

}  // namespace ed
