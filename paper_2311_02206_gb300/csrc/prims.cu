// extern "C" entry points of include/hisa_prims.h: the engine's kernels run
// once on caller buffers, with a throw-away DevState describing them.
#include <cstring>
#include <vector>

#include "hisa_prims.h"
#include "kernels.cuh"

namespace hisa {
namespace {

struct Prim {
  cudaStream_t s;
  DevState h{};
  DevState* d = nullptr;
  std::vector<void*> owned;
  int next = 0;
  Grid g;
  cudaError_t err = cudaSuccess;

  explicit Prim(void* stream) : s(static_cast<cudaStream_t>(stream)) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    g.sms = sms;
    g.radix = sms * 3;
    g.setop = sms * 5;
    g.join = sms * 4;
    g.small = sms * 4;
    void* p = nullptr;
    err = cudaMallocAsync(&p, sizeof(DevState), s);
    d = static_cast<DevState*>(p);
  }
  ~Prim() {
    for (void* p : owned) cudaFreeAsync(p, s);
    if (d) cudaFreeAsync(d, s);
  }
  // a slot over caller memory
  int wrap(const void* p, uint64_t cap, uint64_t cnt) {
    const int id = next++;
    h.buf[id] = {const_cast<void*>(p), cap};
    h.cnt[id] = cnt;
    return id;
  }
  // a slot over fresh scratch
  int scratch(uint64_t elems, int elem_bytes) {
    void* p = nullptr;
    if (err == cudaSuccess) err = cudaMallocAsync(&p, std::max<uint64_t>(elems, 1) * elem_bytes, s);
    if (p) owned.push_back(p);
    return wrap(p, elems, 0);
  }
  int count() { return next++; }
  void zero(int id, uint64_t bytes) {
    if (err == cudaSuccess) err = cudaMemsetAsync(h.buf[id].ptr, 0, bytes, s);
  }
  hisa_status upload() {
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? HISA_ERR_OOM : HISA_ERR_CUDA;
    err = cudaMemcpyAsync(d, &h, sizeof(DevState), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);   // &h is pageable: keep it alive
    return err == cudaSuccess ? HISA_OK : HISA_ERR_CUDA;
  }
  hisa_status download() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return HISA_ERR_CUDA;
    e = cudaMemcpyAsync(&h, d, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HISA_ERR_CUDA;
    if (h.error == kDevTimeout) return HISA_ERR_DEVICE_TIMEOUT;
    if (h.error) return HISA_ERR_CUDA;
    return HISA_OK;
  }
};

template <typename K>
int passes_for(int key_bits) {
  if (key_bits <= 0 || key_bits > int(sizeof(K) * 8)) key_bits = int(sizeof(K) * 8);
  return (key_bits + 7) / 8;
}

// Radix sort of slot `in` into slot `out` through slot `tmp` (P passes; the last
// one writes `out`).  Histogram of all passes first.
template <typename K>
void sort_into(Prim& P, int in, int out, int tmp, int cnt, int passes) {
  const int hist = P.scratch(8 * 256, 8);
  P.zero(hist, 8 * 256 * 8);
  const uint64_t n = P.h.cnt[cnt];
  const uint64_t tiles = (n + radix_tile<K>() - 1) / radix_tile<K>();
  const int status = P.scratch(tiles * 256 + 1, 8);
  P.zero(status, (tiles * 256 + 1) * 8);
  if (P.upload()) return;
  RadixHistArgs ha{P.d, in, cnt, hist, passes, 0};
  launch_radix_hist<K>(ha, P.g, P.s);
  int src = in;
  for (int p = 0; p < passes; ++p) {
    const int dstb = ((passes - 1 - p) % 2 == 0) ? out : tmp;
    RadixPassArgs a{P.d, src, dstb, cnt, hist, status, p, 8 * p, 1, 0, 0};
    launch_radix_pass<K>(a, P.g, P.s);
    src = dstb;
  }
}

template <typename K>
hisa_status sort_t(const void* in, void* out, uint64_t n, int key_bits, void* stream) {
  if (n == 0) return HISA_OK;
  Prim P(stream);
  const int a = P.wrap(in, n, n);
  const int o = P.wrap(out, n, 0);
  const int t = P.scratch(n, sizeof(K));
  sort_into<K>(P, a, o, t, a, passes_for<K>(key_bits));
  return P.download();
}

template <typename K>
hisa_status sort_unique_t(const void* in, void* out, uint64_t n, uint64_t* n_out, int key_bits, void* stream) {
  *n_out = 0;
  if (n == 0) return HISA_OK;
  Prim P(stream);
  const int a = P.wrap(in, n, n);
  const int o = P.wrap(out, n, 0);
  const int t = P.scratch(n, sizeof(K));
  const int sorted = P.scratch(n, sizeof(K));
  sort_into<K>(P, a, sorted, t, a, passes_for<K>(key_bits));
  // unique = difference against an empty full
  const int empty = P.wrap(nullptr, 0, 0);
  const uint64_t tiles = (n + setop_tile<K>() - 1) / setop_tile<K>() + 1;
  const int split = P.scratch(tiles + 1, 8);
  const int status = P.scratch(tiles + 1, 8);
  P.zero(status, (tiles + 1) * 8);
  const int scnt = P.count();
  P.h.cnt[scnt] = n;
  P.h.cnt[o] = 0;
  hisa_status s = P.upload();
  if (s) return s;
  SetopArgs u{P.d, empty, empty, sorted, scnt, split, status, o, o, -1, -1, 2, 0, 1};
  launch_setop<K>(u, P.g, P.s);
  s = P.download();
  if (s) return s;
  *n_out = P.h.cnt[o];
  return HISA_OK;
}

template <typename K>
hisa_status diff_merge_t(const void* full, uint64_t nf, const void* fresh, uint64_t nn, void* dout, uint64_t dcap,
                         void* fout, uint64_t fcap, uint64_t* n_delta, void* stream) {
  *n_delta = 0;
  if (nn == 0) {   // nothing new: delta is empty and full' is a copy of full
    if (fout && nf) {
      if (fcap < nf) return HISA_ERR_CAPACITY;
      if (cudaMemcpyAsync(fout, full, nf * sizeof(K), cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) !=
              cudaSuccess ||
          cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return HISA_ERR_CUDA;
    }
    return HISA_OK;
  }
  Prim P(stream);
  const int A = P.wrap(full, nf, nf);
  const int B = P.wrap(fresh, nn, nn);
  const int D = P.wrap(dout, dcap, 0);
  const int F = fout ? P.wrap(fout, fcap, 0) : -1;
  const uint64_t tiles = (nf + nn + setop_tile<K>() - 1) / setop_tile<K>() + 1;
  const int split = P.scratch(tiles + 1, 8);
  const int status = P.scratch(tiles + 1, 8);
  P.zero(status, (tiles + 1) * 8);
  hisa_status s = P.upload();
  if (s) return s;
  SetopArgs u{P.d, A, A, B, B, split, status, D, D, F, F, 2, 0, 1};
  launch_setop<K>(u, P.g, P.s);
  if ((s = P.download())) return s;
  *n_delta = P.h.cnt[D];
  if (P.h.overflow) return HISA_ERR_CAPACITY;
  return HISA_OK;
}

template <typename K>
hisa_status join_t(const void* outer, uint64_t no, const void* inner, uint64_t ni, int b, int ocol, int p0, int p1,
                   int neq, void* out, uint64_t cap, uint64_t* n_out, void* stream) {
  *n_out = 0;
  Prim P(stream);
  const int O = P.wrap(outer, no, no);
  const int I = P.wrap(inner, ni, ni);
  const int R = P.wrap(out, cap, 0);
  // run index over the inner relation
  const int runs = P.count();
  hisa_status s = P.upload();
  if (s) return s;
  RunsArgs ra{P.d, I, I, b, runs, 0};
  launch_count_runs<K>(ra, P.g, P.s);
  if ((s = P.download())) return s;
  uint64_t tcap = 16;
  while (double(tcap) * 0.8 < double(P.h.cnt[runs])) tcap <<= 1;
  const int T = P.scratch(tcap, 16);
  P.zero(T, tcap * 16);
  const int offs = P.scratch(no + 1, 8);
  const int jst = P.scratch(no / kJoinTile + 2, 8);
  P.zero(jst, (no / kJoinTile + 2) * 8);
  const int total = P.count();
  if ((s = P.upload())) return s;
  IndexArgs ia{P.d, I, I, T, b, -1, 0};
  launch_index<K>(ia, P.g, P.s);
  JoinArgs j{};
  j.st = P.d;
  j.outer_buf = O;
  j.outer_cnt = O;
  j.has_inner = 1;
  j.inner_buf = I;
  j.inner_cnt = I;
  j.table_buf = T;
  j.b = b;
  j.outer_kcol = ocol;
  j.proj0 = p0;
  j.proj1 = p1;
  if (neq) {
    j.nfilt = 1;
    j.fop[0] = kFiltNeq;
    j.fa[0] = (neq - 1) / 4;
    j.fb[0] = (neq - 1) % 4;
  }
  j.offs_buf = offs;
  j.status_buf = jst;
  j.out_buf = R;
  j.out_cnt = R;
  j.total_cnt = total;
  j.hist_buf = -1;
  j.ctr = 0;
  j.skip_mask = 1;
  j.stage_bit = 0;
  // the write partition needs the total: count first, size `starts`, then write
  CtlArgs c{};
  c.st = P.d;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, 0, 0};
  launch_ctl(c, P.s);
  launch_join_count<K>(j, P.g, P.s);
  if ((s = P.download())) return s;
  const uint64_t tot = P.h.cnt[total];
  *n_out = tot;
  if (P.h.overflow) return HISA_ERR_CAPACITY;
  j.starts_buf = P.scratch(tot / kJoinChunk + 2, 8);
  if ((s = P.upload())) return s;
  launch_join_write<K>(j, P.g, P.s);
  return P.download();
}

}  // namespace
}  // namespace hisa

using namespace hisa;

extern "C" {

hisa_status hisa_sort_codes(const void* in, void* out, uint64_t n, int key_bytes, int key_bits, void* stream) {
  if ((!in || !out) && n) return HISA_ERR_INVALID_ARG;
  if (key_bytes == 4) return sort_t<uint32_t>(in, out, n, key_bits, stream);
  if (key_bytes == 8) return sort_t<uint64_t>(in, out, n, key_bits, stream);
  return HISA_ERR_INVALID_ARG;
}

hisa_status hisa_sort_unique_codes(const void* in, void* out, uint64_t n, uint64_t* n_out, int key_bytes,
                                   int key_bits, void* stream) {
  if (!n_out || ((!in || !out) && n)) return HISA_ERR_INVALID_ARG;
  if (key_bytes == 4) return sort_unique_t<uint32_t>(in, out, n, n_out, key_bits, stream);
  if (key_bytes == 8) return sort_unique_t<uint64_t>(in, out, n, n_out, key_bits, stream);
  return HISA_ERR_INVALID_ARG;
}

hisa_status hisa_difference_merge(const void* full, uint64_t n_full, const void* fresh, uint64_t n_new,
                                  void* delta_out, uint64_t delta_cap, void* full_out, uint64_t full_cap,
                                  uint64_t* n_delta, int key_bytes, void* stream) {
  if (!n_delta || (!full && n_full) || (!fresh && n_new) || (!delta_out && delta_cap)) return HISA_ERR_INVALID_ARG;
  if (key_bytes == 4)
    return diff_merge_t<uint32_t>(full, n_full, fresh, n_new, delta_out, delta_cap, full_out, full_cap, n_delta, stream);
  if (key_bytes == 8)
    return diff_merge_t<uint64_t>(full, n_full, fresh, n_new, delta_out, delta_cap, full_out, full_cap, n_delta, stream);
  return HISA_ERR_INVALID_ARG;
}

hisa_status hisa_join_codes(const void* outer, uint64_t n_outer, const void* inner, uint64_t n_inner, int b,
                            int outer_col, int proj0, int proj1, int neq, void* out, uint64_t out_cap,
                            uint64_t* n_out, int key_bytes, void* stream) {
  if (!n_out || b < 1 || b > 32 || outer_col < 0 || outer_col > 1 || proj0 < 0 || proj0 > 3 || proj1 < 0 ||
      proj1 > 3 || neq < 0 || neq > 16 || (!outer && n_outer) || (!inner && n_inner))
    return HISA_ERR_INVALID_ARG;
  if (key_bytes == 4 && 2 * b > 32) return HISA_ERR_INVALID_ARG;
  if (key_bytes == 4)
    return join_t<uint32_t>(outer, n_outer, inner, n_inner, b, outer_col, proj0, proj1, neq, out, out_cap, n_out, stream);
  if (key_bytes == 8)
    return join_t<uint64_t>(outer, n_outer, inner, n_inner, b, outer_col, proj0, proj1, neq, out, out_cap, n_out, stream);
  return HISA_ERR_INVALID_ARG;
}

}  // extern "C"
