/* hisa_prims.h -- the HISA building blocks as single C-ABI calls.
 *
 * Each call runs one step of the semi-naive hot path on caller-owned device
 * buffers, so it can be checked or timed on its own:
 *   hisa_sort_codes          the sorted data array (Section 4.2 "Construction",
 *                            Algorithm 1) as an LSD radix sort of packed codes;
 *   hisa_sort_unique_codes   sort plus removal of adjacent duplicates (Section
 *                            4.2 "Deduplication");
 *   hisa_difference_merge    delta = distinct(new) \ full and full' = full U
 *                            delta (Section 5.1 "Populating delta" and
 *                            "Merging Full with Delta"; Section 4.2 "Merge");
 *   hisa_join_codes          the run index over the inner relation (Section
 *                            4.3, Algorithm 2) and the binary join of
 *                            Algorithm 3 with a projection.
 *
 * Codes: a tuple (c0, c1) of a binary relation is the unsigned integer
 * (c0 << b) | c1 (b = domain bits, 1..32), 4 bytes wide when 2b <= 32 and 8
 * bytes otherwise (key_bytes).  Unsigned order of codes is lexicographic
 * order of tuples.
 *
 * All pointers are device pointers on the current CUDA device; sizes are host
 * values; work runs on `stream` (a cudaStream_t, NULL = legacy default).
 * Each call allocates its scratch with cudaMallocAsync on `stream`, frees it
 * before returning, and synchronises `stream` when it returns a size.  The
 * caller owns every buffer passed in.  Returns HISA_OK or a negative
 * hisa_status (see hisa.h); output buffers that are too small give
 * HISA_ERR_CAPACITY with the needed size stored in the size output.
 */
#ifndef HISA_PRIMS_H_
#define HISA_PRIMS_H_

#include <stdint.h>

#include "hisa.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Sorts n codes (key_bytes 4 or 8; only the low key_bits bits may be set)
 * from `in` into `out` in ascending order.  `in` is not modified; `in` and
 * `out` must not overlap.  Errors: INVALID_ARG, OOM, CUDA. */
hisa_status hisa_sort_codes(const void* in, void* out, uint64_t n, int key_bytes, int key_bits, void* stream);

/* Sorts n codes and keeps one copy of each distinct code: out[0 .. *n_out)
 * ascending.  `out` needs room for n codes.  Synchronises `stream`. */
hisa_status hisa_sort_unique_codes(const void* in, void* out, uint64_t n, uint64_t* n_out, int key_bytes,
                                   int key_bits, void* stream);

/* full: n_full sorted distinct codes; fresh: n_new sorted codes (repeats
 * allowed).  Writes delta = distinct(fresh) \ full (ascending) into
 * delta_out[0 .. *n_delta) and, unless full_out is NULL, full U delta
 * (ascending) into full_out[0 .. n_full + *n_delta).  Capacities are in codes.
 * Errors: CAPACITY (*n_delta holds the needed delta size), INVALID_ARG, OOM,
 * CUDA.  Synchronises `stream`. */
hisa_status hisa_difference_merge(const void* full, uint64_t n_full, const void* fresh, uint64_t n_new,
                                  void* delta_out, uint64_t delta_cap, void* full_out, uint64_t full_cap,
                                  uint64_t* n_delta, int key_bytes, void* stream);

/* Join of outer codes (any order) with inner codes (sorted ascending, distinct)
 * on outer column `outer_col` (0 or 1) == inner column 0: for every outer
 * tuple (o0, o1) and inner tuple (k, x) with o[outer_col] == k, one result
 * (s(proj0), s(proj1)) where source 0 = o0, 1 = o1, 2 = k, 3 = x.  Optional
 * filter `neq` (0 = none, else 1 + 4 * a + b: require s(a) != s(b)).  Results
 * are written in outer order, each outer tuple's results in inner order, as
 * codes (s(proj0) << b) | s(proj1) into out[0 .. *n_out) (capacity out_cap).
 * b = domain bits of all three code arrays.  Errors: CAPACITY (*n_out holds
 * the needed size), INVALID_ARG, OOM, CUDA.  Synchronises `stream`. */
hisa_status hisa_join_codes(const void* outer, uint64_t n_outer, const void* inner, uint64_t n_inner, int b,
                            int outer_col, int proj0, int proj1, int neq, void* out, uint64_t out_cap,
                            uint64_t* n_out, int key_bytes, void* stream);

/* ---- variant that allocates nothing ---------------------------------------------
 *
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory while they run this step (for instance inside a
 * stream capture whose mode forbids allocation calls, on a real-time or
 * signal-safe path that must not enter an allocator, or under a device-memory
 * budget fixed in advance).
 *
 * hisa_difference_merge_noalloc computes exactly what hisa_difference_merge
 * computes, with the same arguments, outputs and errors, but calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch (tile splits,
 * look-back words, control block) lives in one 1 MiB array that the library
 * reserves on every GPU that loads it and holds until the process exits.
 *   - Size limit: n_full + n_new <= HISA_NOALLOC_MAX_CODES (2^26 codes);
 *     larger inputs return HISA_ERR_TOO_LARGE before any GPU work.
 *   - The first call on a device looks up the array's device address with that
 *     device current (cudaGetSymbolAddress); make that first call before any
 *     stream capture that includes this step.
 *   - All calls share the array, which keeps the last call's contents; each
 *     call clears what must start at zero.  Calls whose GPU work overlaps
 *     (other streams or host threads without ordering) race on the array and
 *     give wrong results: order them on one stream.
 *   - Synchronises `stream` to return *n_delta. */
#define HISA_NOALLOC_MAX_CODES (1ull << 26)
#define HISA_ERR_TOO_LARGE (-10) /* input larger than a fixed maximum size */
hisa_status hisa_difference_merge_noalloc(const void* full, uint64_t n_full, const void* fresh, uint64_t n_new,
                                          void* delta_out, uint64_t delta_cap, void* full_out, uint64_t full_cap,
                                          uint64_t* n_delta, int key_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HISA_PRIMS_H_ */
