// Reading an append-only full in lexicographic order without a sort: the
// read side of the sorted levels the grouped bitmap join appends
// (dense.cuh).
#pragma once
#include "dense.cuh"

namespace hisa {

// Reading an append-only full stored column-swapped ((c1, c0): REACH keeps
// the target first) in the declared lexicographic order without sorting it:
// the relation is transposed into a bit matrix M[c0][c1] (2^b rows of 2^b
// bits), whose rows are then counted, scanned and written out in order.
//   transpose: a CTA per block of 16 stored group values t sets, in a shared
//              tile of 2^b 16-bit columns, bit k of column f for every (t0 +
//              k, f) in any level, then stores the tile's columns into M
//              (one 16-bit entry per row); full is read once
//   count:     a warp per row: its population count
//   scan:      one CTA: counts -> row offsets
//   emit:      a CTA per row: its set bits, in order, decoded at the row's
//              offset (coalesced), so a read into page-locked host columns
//              runs at the host link's rate
// M holds 2^(2b) bits: used for b <= 16 (512 MB), where the tile fits in
// shared memory (2^b x 2 bytes).
struct LevelsTransposeArgs {
  DevState* st;
  int full_buf, lvidx_buf, nlv_cnt;
  int b;
  uint32_t* m;        // 2^(2b) bits, row-major (row = c0)
  uint64_t* rowcnt;   // 2^b + 1
  uint32_t* out0;
  uint32_t* out1;
};

template <typename K>
__global__ void __launch_bounds__(1024) k_levels_transpose(LevelsTransposeArgs a) {
  extern __shared__ __align__(16) uint32_t s_tile[];   // 2^(b-1) words: column f in half f & 1 of word f >> 1
  __shared__ uint64_t s_r0[1024], s_r1[1024];          // run bounds of (value k, level l): [k * 64 + l]
  DevState* st = a.st;
  const uint64_t ng = 1ull << a.b, nk1 = ng + 1, ntb = ng / 16, tw = ng / 2;
  const uint64_t nlv = st->cnt[a.nlv_cnt];
  const uint64_t* lvidx = static_cast<const uint64_t*>(st->buf[a.lvidx_buf].ptr);
  const K* fl = static_cast<const K*>(st->buf[a.full_buf].ptr);
  const uint32_t vmask = uint32_t(ng - 1);
  uint16_t* m16 = reinterpret_cast<uint16_t*>(a.m);
  for (uint64_t tb = blockIdx.x; tb < ntb; tb += gridDim.x) {
    for (uint64_t j = threadIdx.x; j < tw; j += blockDim.x) s_tile[j] = 0;
    __syncthreads();
    for (uint64_t l0 = 0; l0 < nlv; l0 += 64) {
      // the run bounds of the block's 16 values in up to 64 levels, one per thread
      const int nl = int(min(uint64_t(64), nlv - l0));
      {
        const int k = threadIdx.x >> 6, l = threadIdx.x & 63;
        if (l < nl) {
          const uint64_t t = tb * 16 + k, lv = l0 + l;
          s_r0[threadIdx.x] = lvidx[lv * nk1 + t];
          s_r1[threadIdx.x] = lvidx[lv * nk1 + t + 1];
        }
      }
      __syncthreads();
      for (int k = 0; k < 16; ++k)
        for (int l = 0; l < nl; ++l) {
          const uint64_t r0 = s_r0[k * 64 + l], r1 = s_r1[k * 64 + l];
          for (uint64_t i0 = r0 + threadIdx.x; i0 < r1; i0 += 4 * uint64_t(blockDim.x)) {
            uint32_t f[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint64_t i = i0 + uint64_t(u) * blockDim.x;
              f[u] = i < r1 ? uint32_t(fl[i]) & vmask : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (f[u] != 0xFFFFFFFFu) atomicOr(&s_tile[f[u] >> 1], 1u << ((f[u] & 1) * 16 + k));
          }
        }
      __syncthreads();
    }
    for (uint64_t f = threadIdx.x; f < ng; f += blockDim.x)
      m16[f * ntb + tb] = uint16_t(s_tile[f >> 1] >> ((f & 1) * 16));
    __syncthreads();
  }
}

// Transpose of a full kept as a bit matrix (row = stored first column) into
// M (row = declared first column): a CTA per tile of 256 x 256 bits; each
// warp loads 32 rows x 8 words (32 contiguous bytes per row), transposes its
// eight 32 x 32-bit blocks with five shuffle-and-mask stages, and the tile is
// written back through shared memory as 256 rows x 8 words.
struct MatrixTransposeArgs {
  const uint32_t* src;   // 2^(2b) bits, row-major
  uint32_t* dst;         // 2^(2b) bits, row-major, dst[c][r] = src[r][c]
  int b;
};
__device__ __forceinline__ uint32_t transpose32_lane(uint32_t x) {
  // lane r holds row r of a 32 x 32 bit block (bit c = column c); returns
  // row r of the transposed block
  const int lane = threadIdx.x & 31;
  const uint32_t lo[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~lo[s]) | ((y & ~lo[s]) >> j)) : ((x & lo[s]) | ((y & lo[s]) << j));
  }
  return x;
}
static __global__ void __launch_bounds__(256) k_matrix_transpose(MatrixTransposeArgs a) {
  __shared__ uint32_t s_t[256][9];   // [transposed row][word], padded
  const uint64_t n = 1ull << a.b, nw = n / 32, tiles = n / 256;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint64_t t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
    const uint64_t tr = t / tiles, tc = t % tiles;   // source rows [256 tr, +256), columns [256 tc, +256)
    const uint32_t* srow = a.src + (tr * 256 + warp * 32 + lane) * nw + tc * 8;
    uint32_t w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) w[u] = srow[u];
#pragma unroll
    for (int u = 0; u < 8; ++u) s_t[u * 32 + lane][warp] = transpose32_lane(w[u]);
    __syncthreads();
    // transposed row R = 256 tc + r holds, in words 8 tr .. 8 tr + 7, the bits of source rows 256 tr ..
    const int r = threadIdx.x;
    uint32_t* drow = a.dst + (tc * 256 + r) * nw + tr * 8;
#pragma unroll
    for (int u = 0; u < 8; ++u) drow[u] = s_t[r][u];
    __syncthreads();
  }
}

template <typename K>
__global__ void k_rows_count(LevelsTransposeArgs a) {
  const uint64_t ng = 1ull << a.b, nw = ng >= 32 ? ng / 32 : 1;   // (b < 5: one word per row)
  const int lane = threadIdx.x & 31;
  for (uint64_t r = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5; r < ng;
       r += (uint64_t(gridDim.x) * blockDim.x) >> 5) {
    const uint32_t* row = a.m + r * nw;
    uint32_t c = 0;
    for (uint64_t j = lane; j < nw; j += 32) c += __popc(row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) a.rowcnt[r] = c;
  }
}

template <typename K>
__global__ void __launch_bounds__(1024) k_rows_scan(LevelsTransposeArgs a) {
  __shared__ uint64_t s_scan[33];
  const uint64_t ng = 1ull << a.b;
  const uint64_t total = cta_scan_inplace(a.rowcnt, ng, s_scan);
  if (threadIdx.x == 0) a.rowcnt[ng] = total;
}

template <typename K>
__global__ void __launch_bounds__(kDenseThreads) k_rows_emit(LevelsTransposeArgs a) {
  constexpr int nwarps = kDenseThreads / 32;
  __shared__ uint32_t s_stage[nwarps][32 * 32];
  __shared__ uint32_t s_wtot[nwarps];
  const uint64_t ng = 1ull << a.b;
  const int nwords = ng >= 32 ? int(ng / 32) : 1;
  const int wrange = (nwords + nwarps - 1) / nwarps;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int w0 = min(nwords, warp * wrange), w1 = min(nwords, w0 + wrange);
  for (uint64_t r = blockIdx.x; r < ng; r += gridDim.x) {
    const uint32_t* row = a.m + r * uint64_t(nwords);
    if (a.rowcnt[r + 1] == a.rowcnt[r]) continue;   // uniform across the CTA
    uint32_t c = 0;
    for (int j = w0 + lane; j < w1; j += 32) c += __popc(row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) s_wtot[warp] = c;
    __syncthreads();
    uint64_t base = a.rowcnt[r];
    for (int w = 0; w < warp; ++w) base += s_wtot[w];
    for (int j0 = w0; j0 < w1; j0 += 32) {
      const int j = j0 + lane;
      const uint32_t bits = j < w1 ? row[j] : 0u;
      const uint32_t pc = __popc(bits);
      uint32_t incl = pc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (tot == 0) continue;
      uint32_t pos = incl - pc;
      uint32_t rest = bits;
      while (rest) {
        const int t = __ffs(rest) - 1;
        rest &= rest - 1;
        s_stage[warp][pos++] = uint32_t(j) * 32u + uint32_t(t);
      }
      __syncwarp();
      for (uint32_t i = lane; i < tot; i += 32) {
        a.out0[base + i] = uint32_t(r);
        a.out1[base + i] = s_stage[warp][i];
      }
      __syncwarp();
      base += tot;
    }
    __syncthreads();   // s_wtot is rewritten by the next row
  }
}

}  // namespace hisa
