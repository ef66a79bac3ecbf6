// hisa_difference_merge_noalloc: the set-difference + merge step for callers
// that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync (or any
// allocating library call) is not allowed or not safe -- a host framework that
// owns all device memory and lends this library only the inputs and outputs, a
// real-time path that must not enter an allocator (an allocation can wait on
// other work or fail when memory is fragmented), or a program that runs under
// a device-memory budget handed out up front.  Such a caller still passes its
// own input and output buffers; only the kernels' scratch (the merge-path tile
// splits, the look-back words and the kernels' control block) has to come from
// somewhere, and here it comes from one array reserved when the library is
// loaded.  The call reads the delta size back to the host, so it synchronises
// the caller's stream before it returns.
//
// The scratch is the file-scope array below (1 MiB).  Every GPU that loads the
// library holds that array until the process exits.  All calls share it and it
// keeps what the last call left there; the parts that must start at zero (the
// look-back words and the control block) are cleared by each call.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads, without ordering between them) race on the array and give wrong
// results: order them on one stream or serialise them.
#include <cstring>
#include <mutex>

#include "hisa_prims.h"
#include "setops.cuh"

namespace hisa {
namespace {

constexpr uint64_t kNoallocScratchBytes = 1ull << 20;
constexpr uint64_t kStateBytes = (sizeof(DevState) + 255) & ~uint64_t(255);
constexpr int kMaxDevices = 64;

// Tiles of the merged sequence at the size limit, for the smaller tile (64-bit codes).
constexpr uint64_t kMaxTiles = HISA_NOALLOC_MAX_CODES / setop_tile<uint64_t>() + 1;
static_assert(kStateBytes + (2 * kMaxTiles + 1) * 8 <= kNoallocScratchBytes, "scratch array too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device, with that device current, and reused.
hisa_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HISA_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return HISA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HISA_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HISA_OK;
}

struct NoallocSetup {
  DevState* st;
  const void* full;
  uint64_t n_full;
  const void* fresh;
  uint64_t n_new;
  void* delta_out;
  uint64_t delta_cap;
  void* full_out;
  uint64_t full_cap;
  uint64_t* splits;
  uint64_t* status;
  uint64_t tiles;
};

// Writes the control block the set-operation kernels read and clears the
// look-back words of the tiles this call uses.
__global__ void k_noalloc_setup(NoallocSetup a) {
  DevState* st = a.st;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->buf[0] = {const_cast<void*>(a.full), a.n_full};
    st->buf[1] = {const_cast<void*>(a.fresh), a.n_new};
    st->buf[2] = {a.splits, a.tiles + 1};
    st->buf[3] = {a.status, a.tiles};
    st->buf[4] = {a.delta_out, a.delta_cap};
    st->buf[5] = {a.full_out, a.full_cap};
    for (int i = 0; i < 6; ++i) {
      st->cnt[i] = 0;
      st->need[i] = 0;
    }
    st->cnt[0] = a.n_full;
    st->cnt[1] = a.n_new;
    st->overflow = 0;
    st->error = 0;
    st->epoch = 1;
    st->tile_ctr[2] = 0;
  }
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.tiles; i += uint64_t(gridDim.x) * blockDim.x)
    a.status[i] = 0;
}

template <typename K>
hisa_status run_noalloc(const void* full, uint64_t nf, const void* fresh, uint64_t nn, void* dout, uint64_t dcap,
                        void* fout, uint64_t fcap, uint64_t* n_delta, cudaStream_t s) {
  void* base = nullptr;
  hisa_status rc = scratch_address(&base);
  if (rc) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HISA_ERR_CUDA;
  const uint64_t tiles = (nf + nn + setop_tile<K>() - 1) / setop_tile<K>();
  NoallocSetup su{};
  su.st = static_cast<DevState*>(base);
  su.full = full;
  su.n_full = nf;
  su.fresh = fresh;
  su.n_new = nn;
  su.delta_out = dout;
  su.delta_cap = dcap;
  su.full_out = fout;
  su.full_cap = fout ? fcap : 0;
  su.splits = reinterpret_cast<uint64_t*>(static_cast<unsigned char*>(base) + kStateBytes);
  su.status = su.splits + (kMaxTiles + 1);
  su.tiles = tiles;
  k_noalloc_setup<<<sms, 256, 0, s>>>(su);
  SetopArgs a{su.st, 0, 0, 1, 1, 2, 3, 4, 4, fout ? 5 : -1, fout ? 5 : -1, 2, 0, 1};
  k_setop_partition<K><<<sms * 4, 256, 0, s>>>(a);
  k_setop<K><<<sms * 4, kSetopThreads, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return HISA_ERR_CUDA;
  // read back the delta size and the status words (plain copy into host memory)
  DevState h;
  if (cudaMemcpyAsync(&h, su.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HISA_ERR_CUDA;
  if (h.error == kDevTimeout) return HISA_ERR_DEVICE_TIMEOUT;
  if (h.error) return HISA_ERR_CUDA;
  *n_delta = h.cnt[4];
  if (h.overflow) return HISA_ERR_CAPACITY;
  return HISA_OK;
}

}  // namespace
}  // namespace hisa

extern "C" hisa_status hisa_difference_merge_noalloc(const void* full, uint64_t n_full, const void* fresh,
                                                     uint64_t n_new, void* delta_out, uint64_t delta_cap,
                                                     void* full_out, uint64_t full_cap, uint64_t* n_delta,
                                                     int key_bytes, void* stream) {
  if (!n_delta || (!full && n_full) || (!fresh && n_new) || (!delta_out && delta_cap)) return HISA_ERR_INVALID_ARG;
  *n_delta = 0;
  if (n_full > HISA_NOALLOC_MAX_CODES || n_new > HISA_NOALLOC_MAX_CODES ||
      n_full + n_new > HISA_NOALLOC_MAX_CODES)
    return HISA_ERR_TOO_LARGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (key_bytes != 4 && key_bytes != 8) return HISA_ERR_INVALID_ARG;
  if (n_new == 0) {   // nothing new: delta is empty and full' is a copy of full
    if (full_out && n_full) {
      if (full_cap < n_full) return HISA_ERR_CAPACITY;
      if (cudaMemcpyAsync(full_out, full, n_full * key_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return HISA_ERR_CUDA;
    }
    return HISA_OK;
  }
  if (key_bytes == 4)
    return hisa::run_noalloc<uint32_t>(full, n_full, fresh, n_new, delta_out, delta_cap, full_out, full_cap, n_delta, s);
  if (key_bytes == 8)
    return hisa::run_noalloc<uint64_t>(full, n_full, fresh, n_new, delta_out, delta_cap, full_out, full_cap, n_delta, s);
  return HISA_ERR_INVALID_ARG;
}
