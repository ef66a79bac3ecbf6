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
  j.starts_buf = P.scratch(tot / kJoinChunkMin + 2, 8);
  if ((s = P.upload())) return s;
  launch_join_write<K>(j, P.g, P.s);
  return P.download();
}

// ---- hash partitioning (multi-GPU scheme) ------------------------------------------------

template <typename K>
__global__ void k_encode_pairs(const uint32_t* c0, const uint32_t* c1, uint64_t n, int b, K* out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    out[i] = (K(c0[i]) << b) | K(c1[i]);
}

template <typename K>
__global__ void k_decode_pairs(const K* in, uint64_t n, int b, uint32_t* c0, uint32_t* c1) {
  const K mask = b >= int(sizeof(K) * 8) ? ~K(0) : ((K(1) << b) - 1);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const K c = in[i];
    c0[i] = uint32_t(c >> b);
    c1[i] = uint32_t(c & mask);
  }
}

template <typename K>
__device__ __forceinline__ uint32_t part_owner(K code, int b, int key_col, uint32_t nparts) {
  const K mask = (K(1) << b) - 1;
  const uint32_t key = key_col == 0 ? uint32_t(code >> b) : uint32_t(code & mask);
  return fmix32(key) % nparts;
}

// Counts per part of block `blockIdx.x`'s contiguous chunk of the codes.
template <typename K>
__global__ void k_part_count(const K* in, uint64_t n, uint64_t chunk, int b, int key_col, uint32_t nparts,
                             uint32_t* bcount) {
  extern __shared__ uint32_t s_pc[];
  for (uint32_t p = threadIdx.x; p < nparts; p += blockDim.x) s_pc[p] = 0;
  __syncthreads();
  const uint64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&s_pc[part_owner(in[i], b, key_col, nparts)], 1u);
  __syncthreads();
  for (uint32_t p = threadIdx.x; p < nparts; p += blockDim.x) bcount[uint64_t(blockIdx.x) * nparts + p] = s_pc[p];
}

// One CTA: each block's first output position per part (parts in order,
// blocks in order within a part) and each part's total.
__global__ void k_part_offsets(const uint32_t* bcount, uint32_t nblocks, uint32_t nparts, uint64_t* off,
                               uint64_t* totals) {
  __shared__ uint64_t s_scan[33];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t p0 = 0; p0 < nparts; p0 += blockDim.x) {
    const uint32_t p = p0 + threadIdx.x;
    uint64_t run = 0;
    if (p < nparts)
      for (uint32_t k = 0; k < nblocks; ++k) {
        off[uint64_t(k) * nparts + p] = run;
        run += bcount[uint64_t(k) * nparts + p];
      }
    uint64_t tot;
    const uint64_t base = s_carry + block_exclusive_sum<uint64_t>(run, s_scan, &tot);
    if (p < nparts) {
      totals[p] = run;
      for (uint32_t k = 0; k < nblocks; ++k) off[uint64_t(k) * nparts + p] += base;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
}

// Each block scatters its chunk to its positions (order within a part and a
// block unspecified: the receiver sorts).
template <typename K>
__global__ void k_part_scatter(const K* in, uint64_t n, uint64_t chunk, int b, int key_col, uint32_t nparts,
                               const uint64_t* off, K* out) {
  extern __shared__ unsigned long long s_po[];
  for (uint32_t p = threadIdx.x; p < nparts; p += blockDim.x) s_po[p] = off[uint64_t(blockIdx.x) * nparts + p];
  __syncthreads();
  const uint64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const K c = in[i];
    out[atomicAdd(&s_po[part_owner(c, b, key_col, nparts)], 1ull)] = c;
  }
}

template <typename K>
hisa_status partition_t(const void* in, uint64_t n, int b, int key_col, uint32_t nparts, void* out, uint64_t* counts,
                        cudaStream_t s) {
  for (uint32_t p = 0; p < nparts; ++p) counts[p] = 0;
  if (n == 0) return HISA_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HISA_ERR_CUDA;
  const uint32_t nblocks = uint32_t(std::max(1, sms * 4));
  const uint64_t chunk = (n + nblocks - 1) / nblocks;
  uint32_t* bcount = nullptr;
  uint64_t *off = nullptr, *totals = nullptr;
  cudaError_t e = cudaMallocAsync(&bcount, size_t(nblocks) * nparts * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&off, size_t(nblocks) * nparts * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&totals, size_t(nparts) * 8, s);
  hisa_status rc = HISA_OK;
  if (e != cudaSuccess) {
    rc = e == cudaErrorMemoryAllocation ? HISA_ERR_OOM : HISA_ERR_CUDA;
  } else {
    k_part_count<K><<<nblocks, 256, nparts * 4, s>>>(static_cast<const K*>(in), n, chunk, b, key_col, nparts, bcount);
    k_part_offsets<<<1, 256, 0, s>>>(bcount, nblocks, nparts, off, totals);
    k_part_scatter<K><<<nblocks, 256, nparts * 8, s>>>(static_cast<const K*>(in), n, chunk, b, key_col, nparts, off,
                                                      static_cast<K*>(out));
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(counts, totals, size_t(nparts) * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = HISA_ERR_CUDA;
  }
  if (bcount) cudaFreeAsync(bcount, s);
  if (off) cudaFreeAsync(off, s);
  if (totals) cudaFreeAsync(totals, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = HISA_ERR_CUDA;
  return rc;
}

__global__ void k_column_max(const uint32_t* a, const uint32_t* b2, uint64_t n, uint32_t* out) {
  uint32_t m = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    m = max(m, max(a[i], b2[i]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---- fault path of the bounded waits -------------------------------------------------

// One of the library's bounded device-side waits, run on a word that nothing
// publishes (or an mbarrier that nothing arrives on, with no copy in flight)
// and a short limit: the wait must run out, record kDevTimeout and return.
__global__ void k_check_bounded_wait(DevState* st, int which, uint32_t limit, uint64_t* status) {
  __shared__ __align__(8) uint64_t mbar;
  constexpr uint32_t epoch = 1;
  constexpr uint64_t tile = 5;   // predecessors 0..4 are never published
  if (which == 0) {
    if (threadIdx.x < 32) lookback_warp(status, tile, 1, epoch, &st->error, limit);
  } else if (which == 1) {
    if (threadIdx.x == 0) {
      lookback_publish(status, tile, 1, 1, epoch);
      lookback_resolve(status, tile, 1, 1, epoch, &st->error, limit);
    }
  } else if (which == 2) {
    if (threadIdx.x == 0) lookback_thread(status, tile, 1, 1, epoch, &st->error, limit);
  } else {
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&mbar, 0, limit)) atomicExch(&st->error, kDevTimeout);
  }
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

hisa_status hisa_check_bounded_wait(int which, uint32_t spin_limit, void* stream) {
  if (which < 0 || which > 3 || spin_limit < 1 || spin_limit > 65536) return HISA_ERR_INVALID_ARG;
  Prim P(stream);
  const int status = P.scratch(16, 8);
  P.zero(status, 16 * 8);
  hisa_status s = P.upload();
  if (s) return s;
  k_check_bounded_wait<<<1, 32, 0, P.s>>>(P.d, which, spin_limit, static_cast<uint64_t*>(P.h.buf[status].ptr));
  return P.download();
}

hisa_status hisa_encode_codes(const uint32_t* c0, const uint32_t* c1, uint64_t n, int b, void* out, int key_bytes,
                              void* stream) {
  if (b < 1 || b > 32 || (key_bytes != 4 && key_bytes != 8) || (key_bytes == 4 && 2 * b > 32) ||
      (n && (!c0 || !c1 || !out)))
    return HISA_ERR_INVALID_ARG;
  if (n == 0) return HISA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = unsigned(std::min<uint64_t>((n + 255) / 256, 152 * 8));
  if (key_bytes == 4) k_encode_pairs<uint32_t><<<grid, 256, 0, s>>>(c0, c1, n, b, static_cast<uint32_t*>(out));
  else k_encode_pairs<uint64_t><<<grid, 256, 0, s>>>(c0, c1, n, b, static_cast<uint64_t*>(out));
  return cudaGetLastError() == cudaSuccess ? HISA_OK : HISA_ERR_CUDA;
}

hisa_status hisa_decode_codes(const void* in, uint64_t n, int b, uint32_t* c0, uint32_t* c1, int key_bytes,
                              void* stream) {
  if (b < 1 || b > 32 || (key_bytes != 4 && key_bytes != 8) || (key_bytes == 4 && 2 * b > 32) ||
      (n && (!in || !c0 || !c1)))
    return HISA_ERR_INVALID_ARG;
  if (n == 0) return HISA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = unsigned(std::min<uint64_t>((n + 255) / 256, 152 * 8));
  if (key_bytes == 4) k_decode_pairs<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t*>(in), n, b, c0, c1);
  else k_decode_pairs<uint64_t><<<grid, 256, 0, s>>>(static_cast<const uint64_t*>(in), n, b, c0, c1);
  return cudaGetLastError() == cudaSuccess ? HISA_OK : HISA_ERR_CUDA;
}

hisa_status hisa_partition_codes(const void* in, uint64_t n, int key_bytes, int b, int key_col, uint32_t nparts,
                                 void* out, uint64_t* counts, void* stream) {
  if (!counts || nparts < 1 || nparts > 1024 || key_col < 0 || key_col > 1 || b < 1 || b > 32 ||
      (key_bytes != 4 && key_bytes != 8) || (key_bytes == 4 && 2 * b > 32) || (n && (!in || !out)))
    return HISA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (key_bytes == 4) return partition_t<uint32_t>(in, n, b, key_col, nparts, out, counts, s);
  return partition_t<uint64_t>(in, n, b, key_col, nparts, out, counts, s);
}

hisa_status hisa_column_max(const uint32_t* c0, const uint32_t* c1, uint64_t n, uint32_t* out, void* stream) {
  if (!out || (n && (!c0 || !c1))) return HISA_ERR_INVALID_ARG;
  *out = 0;
  if (n == 0) return HISA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, 4, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? HISA_ERR_OOM : HISA_ERR_CUDA;
  hisa_status rc = HISA_OK;
  if (cudaMemsetAsync(d, 0, 4, s) != cudaSuccess) rc = HISA_ERR_CUDA;
  if (!rc) {
    const unsigned grid = unsigned(std::min<uint64_t>((n + 255) / 256, 152 * 8));
    k_column_max<<<grid, 256, 0, s>>>(c0, c1, n, d);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(out, d, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = HISA_ERR_CUDA;
  }
  cudaFreeAsync(d, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = HISA_ERR_CUDA;
  return rc;
}

}  // extern "C"
