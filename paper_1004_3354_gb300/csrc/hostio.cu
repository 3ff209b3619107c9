// y = H x for vectors that live in host memory: the end-to-end form of the
// matrix-free H*v (the paper's iterative solver applies H to vectors it holds
// in host memory; here every byte crosses the host link once each way).
//
// n_vec vectors are processed as a pipeline on three streams with two device
// buffers each way: while H*v runs on vector i, vector i + 1 is copied in and
// vector i - 1 is copied out, so the host link carries both directions at
// once and the apply hides behind the copies.  The device buffers and streams
// are made at the first call on a sector and kept until it is destroyed.
#include <algorithm>

#include "ed_internal.h"

namespace ed {

struct HostXfer {
  void* xd[2] = {nullptr, nullptr};
  void* yd[2] = {nullptr, nullptr};
  size_t bytes = 0;
  cudaStream_t s_in = nullptr, s_cmp = nullptr, s_out = nullptr;
  cudaEvent_t h2d[2] = {nullptr, nullptr}, app[2] = {nullptr, nullptr}, d2h[2] = {nullptr, nullptr};
  cudaEvent_t start = nullptr, fin_in = nullptr, fin_cmp = nullptr, fin_out = nullptr;
};

void host_xfer_free(Ctx* c, HostXfer* h) {
  if (!h) return;
  for (int b = 0; b < 2; ++b) {
    dev_free(c, h->xd[b], h->bytes);
    dev_free(c, h->yd[b], h->bytes);
  }
  cudaEvent_t* evs[] = {&h->h2d[0], &h->h2d[1], &h->app[0], &h->app[1], &h->d2h[0], &h->d2h[1],
                        &h->start, &h->fin_in, &h->fin_cmp, &h->fin_out};
  for (auto e : evs)
    if (*e) cudaEventDestroy(*e);
  for (cudaStream_t s : {h->s_in, h->s_cmp, h->s_out})
    if (s) cudaStreamDestroy(s);
  delete h;
}

static int host_xfer_make(Sector* s, HostXfer** out) {
  HostXfer* h = new HostXfer();
  h->bytes = s->dim * elem_bytes(s->prec);
  int st = ED_OK;
  for (int b = 0; b < 2 && st == ED_OK; ++b) {
    st = dev_alloc(s->ctx, &h->xd[b], h->bytes);
    if (st == ED_OK) st = dev_alloc(s->ctx, &h->yd[b], h->bytes);
  }
  cudaError_t e = cudaSuccess;
  for (cudaStream_t* p : {&h->s_in, &h->s_cmp, &h->s_out})
    if (st == ED_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
  cudaEvent_t* evs[] = {&h->h2d[0], &h->h2d[1], &h->app[0], &h->app[1], &h->d2h[0], &h->d2h[1],
                        &h->start, &h->fin_in, &h->fin_cmp, &h->fin_out};
  for (auto p : evs)
    if (st == ED_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(p, cudaEventDisableTiming);
  if (st == ED_OK && e != cudaSuccess) {
    set_error("stream / event creation failed: %s", cudaGetErrorString(e));
    st = ED_ERR_CUDA;
  }
  if (st != ED_OK) {
    host_xfer_free(s->ctx, h);
    return st;
  }
  *out = h;
  return ED_OK;
}

int apply_h_host(Sector* s, HostXfer** hp, uint64_t n_vec, const void* xh, void* yh, cudaStream_t st) {
  if (!xh || !yh) ED_INVALID("NULL host vector");
  if (n_vec == 0) return ED_OK;
  if (!*hp) ED_TRY(host_xfer_make(s, hp));
  HostXfer* h = *hp;
  const size_t bytes = h->bytes;
  const char* xs = static_cast<const char*>(xh);
  char* ys = static_cast<char*>(yh);
  // everything already queued on the caller's stream comes first
  ED_TRY_CUDA(cudaEventRecord(h->start, st));
  ED_TRY_CUDA(cudaStreamWaitEvent(h->s_in, h->start, 0));
  ED_TRY_CUDA(cudaStreamWaitEvent(h->s_cmp, h->start, 0));
  ED_TRY_CUDA(cudaStreamWaitEvent(h->s_out, h->start, 0));
  for (uint64_t i = 0; i < n_vec; ++i) {
    const int b = (int)(i % 2);
    if (i >= 2) ED_TRY_CUDA(cudaStreamWaitEvent(h->s_in, h->app[b], 0));   // vector i-2 has left xd[b]
    ED_TRY_CUDA(cudaMemcpyAsync(h->xd[b], xs + i * bytes, bytes, cudaMemcpyHostToDevice, h->s_in));
    ED_TRY_CUDA(cudaEventRecord(h->h2d[b], h->s_in));
    ED_TRY_CUDA(cudaStreamWaitEvent(h->s_cmp, h->h2d[b], 0));
    if (i >= 2) ED_TRY_CUDA(cudaStreamWaitEvent(h->s_cmp, h->d2h[b], 0));  // y of vector i-2 is out of yd[b]
    ED_TRY(apply_h(s, h->xd[b], h->yd[b], h->s_cmp));
    ED_TRY_CUDA(cudaEventRecord(h->app[b], h->s_cmp));
    ED_TRY_CUDA(cudaStreamWaitEvent(h->s_out, h->app[b], 0));
    ED_TRY_CUDA(cudaMemcpyAsync(ys + i * bytes, h->yd[b], bytes, cudaMemcpyDeviceToHost, h->s_out));
    ED_TRY_CUDA(cudaEventRecord(h->d2h[b], h->s_out));
  }
  // the caller's stream continues once every copy and apply is done
  ED_TRY_CUDA(cudaEventRecord(h->fin_in, h->s_in));
  ED_TRY_CUDA(cudaEventRecord(h->fin_cmp, h->s_cmp));
  ED_TRY_CUDA(cudaEventRecord(h->fin_out, h->s_out));
  ED_TRY_CUDA(cudaStreamWaitEvent(st, h->fin_in, 0));
  ED_TRY_CUDA(cudaStreamWaitEvent(st, h->fin_cmp, 0));
  ED_TRY_CUDA(cudaStreamWaitEvent(st, h->fin_out, 0));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  return ED_OK;
}

}  // namespace ed
