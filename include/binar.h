/*
 * binar.h -- C ABI of libbinar, binar sort on NVIDIA GB300 (sm_103a).
 *
 * Binar sort (W. F. Gilreath, "Binar Sort: A Linear Generalized Sorting
 * Algorithm", arXiv:0811.3448) orders records by the bits of their keys'
 * binary encoding, most significant bit first: each pass splits a sub-array
 * into a lower part (bit 0) and an upper part (bit 1) and recurses into both
 * until the bits run out or a part holds one element ("Algorithm Synopsis",
 * "Operation of Algorithm").  This library runs that recursion on the GPU k
 * bits at a time: every pass splits each live sub-array ("bucket") into 2^k
 * buckets by the next k bits, buckets of at most a cutoff C keys are finished
 * inside one CTA's shared memory, and the rest go on to the next pass.
 *
 * Conventions shared by every call:
 *  - Device pointers are CUDA device addresses; the caller owns all memory.
 *    Keys and payloads must be aligned to their element size (key_bytes,
 *    val_bytes); the workspace must be 16-byte aligned.
 *  - Sorting is in place on the caller's buffers (as the paper's algorithm
 *    is, "Space Analysis"), using a caller-provided workspace of
 *    binar_workspace_bytes() bytes for the out-of-place passes.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  The sort
 *    calls only enqueue work: they never allocate, never synchronise, and can
 *    be captured in a CUDA graph.  The first call on a device performs
 *    one-time host-side set-up (kernel attributes, occupancy queries) and
 *    should come before any stream capture.
 *  - Order: ascending by the key's order-preserving encoding (binar_key_map),
 *    bit 0 = most significant.  Pair sorts are stable: records with equal keys
 *    keep their input order ("Sorting Formalism": the result is the
 *    permutation that orders the keys; among those, the stable one).
 *  - Synchronous errors are returned as binar_status.  Errors found by the
 *    kernels (a look-back wait that timed out, an index outside its bucket, a
 *    full work queue) are written to a status word inside the workspace and
 *    read with binar_workspace_status(); after such an error the output is
 *    unspecified but no write has left the caller's buffers.
 *  - Limits: key_bytes in {4, 8, 16} for every call, and 17 .. 256 for
 *    binar_sort_keys / binar_sort_pairs; val_bytes in {0, 4, 8}; at most
 *    BINAR_MAX_BUCKET_KEYS keys per array or per segment.
 */
#ifndef BINAR_H
#define BINAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BINAR_MAX_BUCKET_KEYS 2147483646LL
#define BINAR_MAX_STRING_BYTES 4096LL

/* Key-to-bits maps ("The Other Universal Property": data is sorted by its
 * encoding -- two's complement integers, IEEE-754 floats, byte strings).
 * Integer and float keys are little-endian machine words. */
typedef enum {
    BINAR_MAP_UNSIGNED = 0, /* unsigned integer of key_bytes bytes (16: 128-bit little-endian) */
    BINAR_MAP_SIGNED = 1,   /* two's complement: sign bit inverted */
    BINAR_MAP_FLOAT = 2,    /* IEEE-754 binary32/64 (key_bytes 4/8): negatives fully inverted,
                               positives with the sign bit set; -0 < +0; NaNs by sign */
    BINAR_MAP_BYTES_BE = 3  /* byte string, byte 0 most significant (memcmp order) */
} binar_key_map;

typedef enum {
    BINAR_OK = 0,
    BINAR_ERR_INVALID_ARG = 1,          /* bad pointer, size, alignment or enum */
    BINAR_ERR_UNSUPPORTED = 2,          /* valid but unsupported shape (e.g. FLOAT with 16 bytes) */
    BINAR_ERR_WORKSPACE_TOO_SMALL = 3,  /* ws_bytes < binar_workspace_bytes() */
    BINAR_ERR_CUDA = 4,                 /* a CUDA runtime call failed */
    BINAR_ERR_DEVICE_TIMEOUT = 5,       /* device: a look-back wait exceeded its time limit */
    BINAR_ERR_DEVICE_BOUNDS = 6,        /* device: an index fell outside its bucket; write skipped */
    BINAR_ERR_QUEUE_OVERFLOW = 7        /* device: a work list exceeded its capacity */
} binar_status;

/* Tuning knobs; a zero field takes the library default.  Pass NULL for all
 * defaults. */
typedef struct {
    int tile_keys;          /* keys per partition tile: 0 or one of the width's two
                               compiled tiles -- 6144 or 4096 (4-byte keys with a
                               payload), 7168 or 4096 (4-byte keys alone), 4096 or
                               2048 (8-byte keys), 2048 or 1024 (16-byte keys);
                               other values return BINAR_ERR_UNSUPPORTED */
    int bits_per_pass;      /* k, key bits consumed per partition pass: 0 (= 8) or
                               4 .. 8 (the in-place mode takes 0 or 1) */
    int small_cutoff;       /* C: buckets of <= C keys are finished in shared memory;
                               2048 .. the finisher capacity: 8192 / 4096 / 2048
                               keys for 4 / 8 / 16-byte keys (0: the capacity, or
                               for 4-byte keys in calls of at most 2^21 keys 4096,
                               6144 or 3072 by the call's size) */
    int ctas_per_sm;        /* persistent CTAs per SM for the partition kernels (0 = max) */
    int64_t lookback_timeout_ns; /* limit on one look-back wait (0 = 1 s) */
    int debug_skip_publish_tile; /* TEST HOOK: if > 0, tile (value-1) of the first partition
                                    pass never publishes its counts, so that successors time
                                    out; the call then reports BINAR_ERR_DEVICE_TIMEOUT */
} binar_config;

/* Bytes of workspace needed to sort n keys (in num_segments segments; 1 for
 * the unsegmented calls) of key_bytes with val_bytes of payload.  The value
 * covers every binar_config choice.  Writes *out; returns binar_status. */
int binar_workspace_bytes(int64_t n, int64_t num_segments, int key_bytes, int val_bytes,
                          size_t *out);

/* Sorts n keys in place ("Operation of Algorithm"; the recursion of
 * "Algorithm Synopsis" run k bits per pass).
 *   d_keys  device pointer to n keys of key_bytes each (read and written)
 *   map     key-to-bits map; must be valid for key_bytes
 *   Keys of 17 .. 256 bytes ("The Other Universal Property": byte strings of
 *   any width; "Recursion Analysis": cost by their length) take BYTES_BE,
 *   UNSIGNED or SIGNED (little-endian integers of that width) and any byte
 *   alignment; they are ordered through the windows of binar_sort_strings
 *   (stable, so the pair form keeps equal keys in input order) and then moved
 *   into that order.
 *   d_ws    device workspace of ws_bytes >= binar_workspace_bytes(n, 1, key_bytes, 0)
 *   cfg     tuning, or NULL
 *   stream  cudaStream_t
 * Returns binar_status; device-side errors via binar_workspace_status(). */
int binar_sort_keys(void *d_keys, int64_t n, int key_bytes, binar_key_map map,
                    void *d_ws, size_t ws_bytes, const binar_config *cfg, void *stream);

/* Sorts n records (key + payload) in place, stably ("Sorting Formalism":
 * records R_i carry keys K_i; equal keys keep their input order).
 *   d_vals  device pointer to n payloads of val_bytes each (moved with their keys)
 * Other arguments as binar_sort_keys; ws_bytes >= binar_workspace_bytes(n, 1,
 * key_bytes, val_bytes). */
int binar_sort_pairs(void *d_keys, void *d_vals, int64_t n, int key_bytes, binar_key_map map,
                     int val_bytes, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                     void *stream);

/* Bytes of workspace binar_sort_inplace needs for n keys of key_bytes with
 * val_bytes of payload and the config's cutoff (cfg may be NULL).  About one
 * bit per key plus a few words per bucket, tile and finisher job: for 256M
 * uint32 keys and payloads a few hundred MB, against the 2 GiB second array
 * of the other sorts. */
int binar_inplace_workspace_bytes(int64_t n, int key_bytes, int val_bytes,
                                  const binar_config *cfg, size_t *out);

/* Sorts n keys (and payloads) in place and unstably, as the paper's algorithm
 * does ("Partition Array into Sub-arrays": one bit per pass, misplaced
 * elements exchanged between the lower and the upper sub-array; "Space
 * Analysis": no second array; "Conclusion": unstable).  Every live sub-array
 * of a level is split on its next bit at once: the k-th element with bit 1
 * below the split point is exchanged with the k-th element with bit 0 above
 * it; sub-arrays of at most the cutoff are finished in shared memory and
 * written back in place.  Keys come out in the same order as binar_sort_keys;
 * records with equal keys come out in an unspecified order.
 *   Arguments as binar_sort_pairs (d_vals NULL and val_bytes 0 for keys only);
 *   key_bytes in {4, 8, 16}; cfg may set small_cutoff and the wait limit (tile
 *   and bits per pass are fixed: 1024-key tiles, one bit);
 *   ws_bytes >= binar_inplace_workspace_bytes(n, key_bytes, val_bytes, cfg). */
int binar_sort_inplace(void *d_keys, void *d_vals, int64_t n, int key_bytes, binar_key_map map,
                       int val_bytes, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                       void *stream);

/* Bytes of workspace binar_sort_strings needs for n strings. */
int binar_strings_workspace_bytes(int64_t n, size_t *out);

/* The stable lexicographic order of n byte strings of different lengths
 * ("The Other Universal Property": strings are sorted by their encoding; the
 * paper's cost per string is its length, "Recursion Analysis").  String i is
 * the bytes d_bytes[d_offsets[i] .. d_offsets[i+1]); bytes compare unsigned,
 * the first difference decides, a proper prefix comes first, equal strings
 * keep their input order.
 *   d_bytes    device pointer to the string bytes (read only)
 *   d_offsets  device pointer to n + 1 int64, nondecreasing (8-byte aligned)
 *   max_len    an upper bound on every string's length, <= BINAR_MAX_STRING_BYTES;
 *              the work runs max_len / 15 + 1 window levels, each of which
 *              only touches the strings still tied with another one
 *   d_order    device pointer to n uint32 (4-byte aligned) receiving the order:
 *              d_order[k] = index of the k-th string
 *   d_ws       device workspace of ws_bytes >= binar_strings_workspace_bytes(n)
 * The strings are not moved.  A string longer than max_len is reported as
 * BINAR_ERR_INVALID_ARG through binar_workspace_status (the order is then
 * unspecified).  Returns binar_status; like the sort calls it only enqueues
 * work on `stream`. */
int binar_sort_strings(const void *d_bytes, const int64_t *d_offsets, int64_t n, int64_t max_len,
                       uint32_t *d_order, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                       void *stream);

/* Sorts num_segments independent segments in one call: segment s is
 * [offsets[s], offsets[s+1]) of the key (and payload) arrays.  The segments
 * become the first-level buckets of the recursion ("Algorithm Variants": each
 * part is sorted independently of the others).
 *   d_vals     payloads or NULL (then val_bytes must be 0)
 *   d_offsets  device pointer to num_segments+1 int64, nondecreasing, offsets[0] >= 0,
 *              offsets[num_segments] <= n; each segment <= BINAR_MAX_BUCKET_KEYS keys.
 *              Offsets are read on the device; a decreasing pair is reported as
 *              BINAR_ERR_INVALID_ARG through the status word and that segment is skipped.
 *   ws_bytes   >= binar_workspace_bytes(n, num_segments, key_bytes, val_bytes)
 * Keys outside every segment are not touched.  Keys wider than 16 bytes are
 * not accepted here (BINAR_ERR_UNSUPPORTED). */
int binar_sort_segmented(void *d_keys, void *d_vals, const int64_t *d_offsets,
                         int64_t num_segments, int64_t n, int key_bytes, binar_key_map map,
                         int val_bytes, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                         void *stream);

/* One stable partition pass, out of place ("Partition Array into Sub-arrays"
 * with k bits instead of one; the parallel variant of "Algorithm Variants"
 * splits by leading bits the same way): the n records of d_keys_in/d_vals_in
 * are written to d_keys_out/d_vals_out grouped by the digit formed by bits
 * pos .. pos+bits-1 of each key's encoding (bits past the key read as 0),
 * digit groups in ascending order, input order kept inside each group.
 *   d_offsets  device pointer to 2^bits + 1 int64 receiving the group bounds, or NULL
 *   bits       0 (= 8) or 1 .. 8;  0 <= pos < 8 * key_bytes
 *   ws_bytes   >= binar_workspace_bytes(n, 1, key_bytes, val_bytes)
 * Input and output must not overlap. */
int binar_partition_pass(const void *d_keys_in, const void *d_vals_in, void *d_keys_out,
                         void *d_vals_out, int64_t n, int key_bytes, binar_key_map map,
                         int val_bytes, int pos, int bits, int64_t *d_offsets, void *d_ws,
                         size_t ws_bytes, const binar_config *cfg, void *stream);

/* The partition pass of binar_partition_pass without a workspace argument:
 * the library allocates nothing and uses 4 MiB of scratch memory that it
 * declares itself (one fixed array per GPU that loads the library, kept until
 * the process exits).  The paper has no counterpart; this exists for callers
 * that cannot allocate or keep a workspace -- e.g. code that owns all device
 * memory through a fixed pool with a hard budget, or a latency-critical loop
 * that must not call (and synchronise on) cudaMalloc.
 *   Arguments, layout and results as binar_partition_pass.
 *   Limit: n <= 29,173,759 keys of 4 bytes alone, 25,006,079 of 4 bytes
 *   with a payload, 16,670,719 of 8 bytes, 8,335,359 of 16 bytes (the
 *   look-back state of one pass in 4 MiB);
 *   larger n returns BINAR_ERR_WORKSPACE_TOO_SMALL before any work.
 *   The first call on a device looks up the scratch array's device address
 *   (host-side set-up); make that first call before any stream capture.
 *   Every call shares the one scratch array and each call resets what it
 *   needs, so calls that overlap on the GPU (different streams, or threads)
 *   race and must not be issued.  Device-side errors (a wait past its time
 *   limit, an index outside its range) are recorded in the shared scratch and
 *   read with binar_partition_pass_noalloc_status(). */
int binar_partition_pass_noalloc(const void *d_keys_in, const void *d_vals_in, void *d_keys_out,
                                 void *d_vals_out, int64_t n, int key_bytes, binar_key_map map,
                                 int val_bytes, int pos, int bits, int64_t *d_offsets,
                                 void *stream);

/* Status of the most recent binar_partition_pass_noalloc call on this
 * device (each call clears the word when its first kernel runs): waits for
 * `stream`, then reads the status word in the library's scratch array into
 * *out_status (a binar_status, BINAR_OK if no kernel of that call reported an
 * error) and clears it.  Like the pass itself it
 * allocates nothing (the word moves through a host variable).  The paper has
 * no counterpart.  Returns binar_status of the query itself. */
int binar_partition_pass_noalloc_status(void *stream, int *out_status);

/* TEST HOOK for the calls to binar_partition_pass_noalloc that follow (its
 * counterpart of binar_config's debug_skip_publish_tile and
 * lookback_timeout_ns, which that call takes no config for): if
 * skip_publish_tile > 0, tile (skip_publish_tile - 1) never publishes its
 * counts, so that its successors' look-back waits run out after
 * lookback_timeout_ns (0 = 1 s) and the pass records
 * BINAR_ERR_DEVICE_TIMEOUT.  (0, 0) restores the defaults.  Process-wide;
 * negative arguments return BINAR_ERR_INVALID_ARG. */
int binar_partition_pass_noalloc_debug(int skip_publish_tile, int64_t lookback_timeout_ns);

/* Waits for `stream`, then reads the device status word of the workspace
 * into *out_status (a binar_status) and clears it.  Returns binar_status of
 * the query itself. */
int binar_workspace_status(void *d_ws, void *stream, int *out_status);

/* A static, human-readable name for a binar_status value. */
const char *binar_status_string(int status);

/* Per-kernel timing for measurement.  While profiling is on, every kernel
 * the library launches is bracketed by CUDA events on its stream (not
 * allowed during stream capture).  binar_profile_stop() waits for the events,
 * turns profiling off and writes up to `cap` entries, one per kernel name in
 * first-launch order: launches and summed device time. */
typedef struct {
    char name[40];
    int64_t launches;
    double total_ms;
} binar_kernel_stat;

int binar_profile_start(void);
int binar_profile_stop(binar_kernel_stat *out, int cap, int *count);

/* Synthetic input on the device (no counterpart in the paper, which defines
 * no input generator): writes n elements of `elem_bytes` (4, 8 or 16) to
 * d_out, element i taken from SplitMix64 (Steele, Lea and Flood, OOPSLA
 * 2014) used as a counter-based generator:
 *   x(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15),
 *   mix(z): z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
 *           return z ^ z>>31.
 * 4-byte elements are the low 32 bits of x(seed, i), 8-byte elements x(seed, i);
 * 16-byte elements are x(seed, i) then x(seed ^ 0xD1B54A32D192ED03, i), each
 * little-endian.  d_out must be aligned to elem_bytes.  Asynchronous on
 * `stream`; the caller owns d_out.  Returns BINAR_ERR_INVALID_ARG for bad
 * arguments, BINAR_ERR_CUDA if the launch fails. */
int binar_generate(void *d_out, int64_t n, int elem_bytes, uint64_t seed, void *stream);

/* Library version as "major.minor.patch". */
const char *binar_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BINAR_H */
