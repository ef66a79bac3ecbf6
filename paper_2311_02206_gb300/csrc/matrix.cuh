// Full kept as a bit matrix in batched and served runs (many independent
// instances in one fixpoint, codes (instance, c0, c1)).
//
// Row (instance << b) | g holds bit o for every tuple (g, o) of that instance
// in full (stored column order), 2^b bits per row, so each instance owns a
// contiguous block of 2^b rows.  Section 5.1's "populating delta" becomes a
// bit test and "merge" an OR of delta into the rows (k_matrix_codes): no
// sorted full is rewritten per iteration, and retiring an instance is reading
// its block out (k_matrix_extract) and clearing it.
#pragma once
#include "common.cuh"
#include "dense.cuh"
#include "setops.cuh"

namespace hisa {

// Largest matrix a batched run keeps (2^(instance bits + 2b) bits): beyond it
// the run keeps a sorted full.
constexpr uint64_t kBatchMatrixMaxBytes = 64ull << 30;

// delta = unique(new) \ full for a sorted new (repeats allowed): an item is
// kept iff it differs from its predecessor and its bit is clear in full's
// matrix; kept items are compacted in order through a decoupled look-back
// over the tiles (the scheme of k_diff_probe, with the sorted probes of the
// large level replaced by one bit test).
struct MatrixDiffArgs {
  DevState* st;
  int b_buf, b_cnt;        // sorted new
  int out_buf, out_cnt;    // delta, written from 0
  int status_buf;          // u64 [tiles] look-back
  int fbm_buf;             // full's bit matrix
  int b, row_bits;         // domain bits; bits of a row index (instance bits + b)
  int ctr;
  int skip_mask, stage_bit;
};

template <typename K>
__global__ void __launch_bounds__(kDiffThreads) k_matrix_diff(MatrixDiffArgs a) {
  __shared__ K s_b[kDiffTile];
  __shared__ uint64_t s_scan[32];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_tile;
  __shared__ K s_prev;
  __shared__ int s_has_prev;
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t nb = st->cnt[a.b_cnt];
  if (nb == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->cnt[a.out_cnt] = 0;
    return;
  }
  const uint64_t ntiles = (nb + kDiffTile - 1) / kDiffTile;
  if (st->buf[a.status_buf].cap < ntiles) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.status_buf], (unsigned long long)ntiles);
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* B = static_cast<const K*>(st->buf[a.b_buf].ptr);
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr);
  const uint64_t ocap = st->buf[a.out_buf].cap;
  const uint32_t* fbm = static_cast<const uint32_t*>(st->buf[a.fbm_buf].ptr);
  uint64_t* status = static_cast<uint64_t*>(st->buf[a.status_buf].ptr);
  const uint32_t epoch = st->epoch;
  const uint32_t vmask = (1u << a.b) - 1;
  const uint64_t rmask = (1ull << a.row_bits) - 1;
  const uint64_t nwords = a.b >= 5 ? (1ull << (a.b - 5)) : 1;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t b0 = tile * kDiffTile;
    const int nT = int(min(uint64_t(kDiffTile), nb - b0));
    for (int i = tid; i < nT; i += kDiffThreads) s_b[i] = B[b0 + i];
    if (tid == 0) {
      s_has_prev = b0 > 0;
      if (b0 > 0) s_prev = B[b0 - 1];
    }
    __syncthreads();
    const int i0 = tid * kDiffItems;
    const int nmine = max(0, min(kDiffItems, nT - i0));
    K v[kDiffItems];
    uint32_t keep = 0;
    bool hp = i0 > 0 || s_has_prev;
    K prev = i0 > 0 && nmine > 0 ? s_b[i0 - 1] : s_prev;
    uint32_t w[kDiffItems];
#pragma unroll
    for (int k = 0; k < kDiffItems; ++k) {   // every matrix word in flight first
      v[k] = k < nmine ? s_b[i0 + k] : K(0);
      const uint64_t row = (uint64_t(v[k]) >> a.b) & rmask;
      const uint32_t o = uint32_t(v[k]) & vmask;
      w[k] = k < nmine ? fbm[row * nwords + (o >> 5)] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kDiffItems; ++k) {
      if (k >= nmine) break;
      const uint32_t o = uint32_t(v[k]) & vmask;
      if (!(hp && prev == v[k]) && !((w[k] >> (o & 31)) & 1u)) keep |= 1u << k;
      prev = v[k];
      hp = true;
    }
    const uint32_t kept = __popc(keep);
    uint64_t tile_kept;
    const uint64_t kexcl = block_exclusive_sum<uint64_t>(kept, s_scan, &tile_kept);
    if (tid < 32) {
      const uint64_t base = lookback_warp(status, tile, tile_kept, epoch, &st->error);
      if (tid == 0) s_base = base;
    }
    __syncthreads();   // every thread holds its items in registers: s_b takes the kept ones
    int wpos = int(kexcl);
#pragma unroll
    for (int k = 0; k < kDiffItems; ++k)
      if (keep & (1u << k)) s_b[wpos++] = v[k];
    __syncthreads();
    const uint64_t base = s_base;
    for (int i = tid; i < int(tile_kept); i += kDiffThreads)
      if (base + i < ocap) out[base + i] = s_b[i];
    if (tile == ntiles - 1 && tid == 0) {
      const uint64_t n = base + tile_kept;
      st->cnt[a.out_cnt] = n;
      if (n > ocap) {
        atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)n);
        atomicOr(&st->overflow, 1u << a.stage_bit);
      }
    }
    __syncthreads();
  }
}

// Rows [row0, row0 + nrows) of the matrix read out as codes in the stored
// order: every set bit o of row r gives the code (r << b) | o, written at the
// row's offset (the exclusive sum of the rows' counts, which every update of
// the matrix keeps in fcnt).  Three launches: counts, one-CTA scan, emit.
struct MatrixExtractArgs {
  const uint32_t* fbm;
  const uint32_t* fcnt;
  uint64_t row0, nrows;
  int b;
  uint64_t* offs;   // nrows + 1 entries (scratch); offs[nrows] = total
  void* out;        // K codes
  // instance slots whose blocks are read, in this order (device array; null:
  // the rows row0 ..): row i is then row i mod 2^b of block slots[i >> b]
  const uint32_t* slots = nullptr;
  // a standalone block (a transposed copy): rows 0 .. nrows - 1 of fbm are
  // read, counted by popcount (fcnt unused), and written as the codes of
  // rows code_row0 + i
  bool standalone = false;
  uint64_t code_row0 = 0;
};

__device__ __forceinline__ uint64_t extract_row(const MatrixExtractArgs& a, uint64_t i) {
  if (!a.slots) return a.row0 + i;
  return (uint64_t(a.slots[i >> a.b]) << a.b) | (i & ((1ull << a.b) - 1));
}

static __global__ void k_matrix_extract_counts(MatrixExtractArgs a) {
  const uint64_t nw = a.b >= 5 ? (1ull << (a.b - 5)) : 1ull;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.nrows;
       i += uint64_t(gridDim.x) * blockDim.x) {
    if (a.standalone) {
      uint64_t c = 0;
      for (uint64_t j = 0; j < nw; ++j) c += __popc(a.fbm[i * nw + j]);
      a.offs[i] = c;
    } else {
      a.offs[i] = a.fcnt[extract_row(a, i)];
    }
  }
}

static __global__ void __launch_bounds__(1024) k_matrix_extract_scan(MatrixExtractArgs a) {
  __shared__ uint64_t s_scan[33];
  const uint64_t total = cta_scan_inplace(a.offs, a.nrows, s_scan);
  if (threadIdx.x == 0) a.offs[a.nrows] = total;
}

// One CTA per row (rows with no bits are skipped): each warp takes a
// contiguous share of the row's words, counts its bits, and writes its
// codes in order, 32 words per step staged in shared memory.
template <typename K>
__global__ void __launch_bounds__(kDenseThreads) k_matrix_extract(MatrixExtractArgs a) {
  constexpr int nwarps = kDenseThreads / 32;
  __shared__ K s_stage[nwarps][32 * 32];
  __shared__ uint32_t s_wtot[nwarps];
  const int nwords = a.b >= 5 ? (1 << (a.b - 5)) : 1;
  const int wrange = (nwords + nwarps - 1) / nwarps;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int w0 = min(nwords, warp * wrange), w1 = min(nwords, w0 + wrange);
  K* out = static_cast<K*>(a.out);
  for (uint64_t r = blockIdx.x; r < a.nrows; r += gridDim.x) {
    if (a.offs[r + 1] == a.offs[r]) continue;   // uniform across the CTA
    const uint64_t row = a.standalone ? a.code_row0 + r : extract_row(a, r);
    const uint32_t* rw = a.fbm + (a.standalone ? r : row) * uint64_t(nwords);
    uint32_t c = 0;
    for (int j = w0 + lane; j < w1; j += 32) c += __popc(rw[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) s_wtot[warp] = c;
    __syncthreads();
    uint64_t base = a.offs[r];
    for (int w = 0; w < warp; ++w) base += s_wtot[w];
    for (int j0 = w0; j0 < w1; j0 += 32) {
      const int j = j0 + lane;
      const uint32_t bits = j < w1 ? rw[j] : 0u;
      const uint32_t cnt = __popc(bits);
      uint32_t incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (tot == 0) continue;
      uint32_t pos = incl - cnt;
      for (uint32_t rest = bits; rest; rest &= rest - 1)
        s_stage[warp][pos++] = K((row << a.b) | uint64_t(uint32_t(j) * 32u + uint32_t(__ffs(rest) - 1)));
      __syncwarp();
      for (uint32_t i = lane; i < tot; i += 32) out[base + i] = s_stage[warp][i];
      __syncwarp();
      base += tot;
    }
    __syncthreads();   // s_wtot is rewritten by the next row
  }
}

}  // namespace hisa
