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

/* ---- hash partitioning for the multi-GPU scheme ----------------------------------
 *
 * The paper evaluates on one GPU and names a distributed, MPI-style
 * semi-naive evaluation as future work (its conclusion; the scheme of the
 * distributed relational-algebra work it cites): relations hash-partitioned
 * by their join column over the GPUs, every GPU joining its own delta with its
 * own part of the inner relation, one all-to-all per iteration sending each
 * new tuple to the owner of its key, owners deduplicating, differencing and
 * merging locally, and a sum of |delta| over the GPUs as the termination test.
 * These calls are the per-GPU steps around the exchange that the other calls
 * above do not cover (paper_2311_02206_gb300/partitioned.py drives them).
 *
 * hisa_encode_codes: n tuples from two device columns into codes
 * (c0 << b) | c1 in out[0 .. n) (key_bytes 4 needs 2b <= 32).  Errors:
 * INVALID_ARG, CUDA.  Does not synchronise. */
hisa_status hisa_encode_codes(const uint32_t* c0, const uint32_t* c1, uint64_t n, int b, void* out, int key_bytes,
                              void* stream);

/* hisa_decode_codes: codes back into two device columns.  Errors: INVALID_ARG,
 * CUDA.  Does not synchronise. */
hisa_status hisa_decode_codes(const void* in, uint64_t n, int b, uint32_t* c0, uint32_t* c1, int key_bytes,
                              void* stream);

/* hisa_column_max: the largest value of two device columns of n values into
 * the host word *out (0 when n is 0); it fixes the domain bits b.  Errors:
 * INVALID_ARG, OOM, CUDA.  Synchronises `stream`. */
hisa_status hisa_column_max(const uint32_t* c0, const uint32_t* c1, uint64_t n, uint32_t* out, void* stream);

/* hisa_partition_codes: the n codes of `in` grouped by owner into out[0 .. n):
 * first the codes owned by part 0, then part 1, and so on.  The owner of a code
 * is fmix32(v) mod nparts, v its column key_col (0: c0, 1: c1) and fmix32 the
 * MurmurHash3 32-bit finaliser.  Within a part the order is unspecified (the
 * receiving GPU sorts).  counts (host, nparts entries) receives each part's
 * size.  nparts 1..1024; `in` and `out` must not overlap.  Errors: INVALID_ARG,
 * OOM (its scratch: 12 bytes per part and CTA), CUDA.  Synchronises `stream`. */
hisa_status hisa_partition_codes(const void* in, uint64_t n, int key_bytes, int b, int key_col, uint32_t nparts,
                                 void* out, uint64_t* counts, void* stream);

/* ---- fault path of the bounded device-side waits ---------------------------------
 *
 * The paper describes no failure handling; every wait of this library on
 * another CTA (decoupled look-back over earlier tiles) or on the copy engine
 * (the mbarrier of a radix pass's bulk tile copy) gives up after a fixed
 * number of polls, records a timeout in device memory and lets the kernel
 * return, and the host reports HISA_ERR_DEVICE_TIMEOUT instead of hanging.
 * This call runs one of those waits on a word that nothing publishes (or an
 * mbarrier that nothing arrives on, with no copy in flight), cut to
 * spin_limit polls, so that it must run out:
 *   which = 0  the warp-wide look-back of the join, set-operation and
 *              grouped-join scans;
 *           1  the per-digit look-back of a radix pass (publish, then resolve);
 *           2  the single-thread per-digit look-back;
 *           3  the mbarrier wait for a radix pass's tile copy.
 * Returns HISA_ERR_DEVICE_TIMEOUT when the wait ran out and the kernel
 * returned (the expected result), HISA_OK if it did not run out,
 * INVALID_ARG for `which` outside 0..3 or spin_limit outside 1..65536, OOM or
 * CUDA if its 128-byte scratch could not be had.  The stream stays usable.
 * Synchronises `stream`. */
hisa_status hisa_check_bounded_wait(int which, uint32_t spin_limit, void* stream);

/* ---- variant that allocates nothing ---------------------------------------------
 *
 * The paper has no counterpart to this call.  It exists for callers that must
 * not allocate device memory while this step runs: a host framework that owns
 * all device memory and lends the library only its inputs and outputs, a
 * real-time path that must not enter an allocator (an allocation can wait on
 * other work or fail when memory is fragmented), or a program that runs under
 * a device-memory budget handed out in advance.
 *
 * hisa_difference_merge_noalloc computes exactly what hisa_difference_merge
 * computes, with the same arguments, outputs and errors, but calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch (tile splits,
 * look-back words, control block) lives in one 1 MiB array that the library
 * reserves on every GPU that loads it and holds until the process exits.
 *   - Size limit: n_full + n_new <= HISA_NOALLOC_MAX_CODES (2^26 codes);
 *     larger inputs return HISA_ERR_TOO_LARGE before any GPU work.
 *   - The first call on a device looks up the array's device address with that
 *     device current (cudaGetSymbolAddress) and keeps it for later calls; make
 *     that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents; each
 *     call clears what must start at zero.  Calls whose GPU work overlaps
 *     (other streams or host threads without ordering) race on the array and
 *     give wrong results: order them on one stream.
 *   - Reads the delta size back to the host: whenever it issues GPU work it
 *     synchronises `stream` before it returns. */
#define HISA_NOALLOC_MAX_CODES (1ull << 26)
#define HISA_ERR_TOO_LARGE (-10) /* input larger than a fixed maximum size */
hisa_status hisa_difference_merge_noalloc(const void* full, uint64_t n_full, const void* fresh, uint64_t n_new,
                                          void* delta_out, uint64_t delta_cap, void* full_out, uint64_t full_cap,
                                          uint64_t* n_delta, int key_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HISA_PRIMS_H_ */
