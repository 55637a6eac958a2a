/*
 * oracle/binar_oracle.c -- CPU oracle for binar sort.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * this library.  It shares no code, header or table with the CUDA library: it is
 * a plain, slow, obviously correct restatement of what the method computes.
 *
 * Contents (each function cites the passage it follows):
 *   oracle_map_keys          the order-preserving bit string of a key ("The Other
 *                            Universal Property": two's complement, IEEE-754, byte
 *                            strings are sorted by their encoding)
 *   oracle_binar_sort        the paper's in-place binar sort ("Operation of
 *                            Algorithm", four steps; "Illustration of the
 *                            Algorithm"), recursive, unstable
 *   oracle_binar_sort_parallel  the paper's parallel variant ("Algorithm
 *                            Variants": processor p sorts the elements whose
 *                            leading bits spell p), used only for CPU timing
 *   oracle_stable_radix      stable binary radix sort (LSD, one bit per pass):
 *                            the definition-level oracle for record order when
 *                            equal keys must keep their input order ("Sorting
 *                            Formalism": the permutation p with K_p(1) <= ... )
 *   oracle_partition_pass    one stable split of a range into 2^k sub-arrays by
 *                            k bits at bit position pos (the partition step,
 *                            generalised to k bits as in the parallel variant)
 *   oracle_sort_strings      the stable lexicographic order of byte strings of
 *                            different lengths (a proper prefix first)
 *
 * Key layout: n keys of kb bytes each (kb <= 256), as raw bytes.  Integer and
 * float keys are little-endian machine words (any kb for integers; 4, 8 for
 * floats).  BYTES_BE keys are byte strings compared as big-endian bit strings
 * (byte 0 most significant).  Payloads ("records", Sorting Formalism) are vb
 * opaque bytes per key and move with their key.
 *
 * Bit numbering follows the paper's bit extraction (a shift left by the position,
 * then a test of the top bit): position 0 is the most significant
 * bit of the encoding, and a sort over w bits looks at positions 0 .. w-1 (the
 * worked example uses w = 4 on nybbles stored in the high half of a byte).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

enum { MAP_UNSIGNED = 0, MAP_SIGNED = 1, MAP_FLOAT = 2, MAP_BYTES_BE = 3 };
enum { KB_MAX = 256 };   /* widest key: 2048 bits */

/* --------------------------------------------------------------------------
 * Encoding ("The Other Universal Property").
 *
 * key_bit returns bit `pos` (0 = most significant) of the order-preserving
 * encoding of one key, written from the definitions of the encodings:
 *  - unsigned: the binary numeral itself; the most significant byte of a
 *    little-endian word is its last byte.
 *  - signed (two's complement): the sign bit has weight -2^(w-1); inverting it
 *    turns the order of signed values into the order of unsigned numerals.
 *  - float (IEEE-754 sign-magnitude): a positive value orders by its magnitude
 *    bits once the sign bit is set to 1; a negative value orders in reverse of
 *    its magnitude, so every bit is inverted (its sign bit becomes 0).
 *  - byte strings: lexicographic byte order is the order of the big-endian
 *    bit string.
 * ------------------------------------------------------------------------ */
static int key_bit(const uint8_t *key, int kb, int map, int pos)
{
    if (map == MAP_BYTES_BE)
        return (key[pos / 8] >> (7 - pos % 8)) & 1;

    const uint8_t msb_byte = key[kb - 1];
    int b = (key[kb - 1 - pos / 8] >> (7 - pos % 8)) & 1;
    if (map == MAP_SIGNED) {
        if (pos == 0) b = !b;
    } else if (map == MAP_FLOAT) {
        int negative = msb_byte >> 7;
        if (negative) b = !b;
        else if (pos == 0) b = !b;
    }
    return b;
}

/* Writes the encoding of each key as a big-endian byte string of kb bytes.
 * Returns 0, or -1 for an unsupported (kb, map). */
int oracle_map_keys(const uint8_t *keys, uint8_t *mapped, int64_t n, int kb, int map)
{
    if (kb <= 0 || kb > KB_MAX) return -1;
    if (map == MAP_FLOAT && kb != 4 && kb != 8) return -1;
    if (map < 0 || map > 3) return -1;
    for (int64_t i = 0; i < n; i++) {
        const uint8_t *k = keys + i * kb;
        uint8_t *m = mapped + i * kb;
        memset(m, 0, (size_t)kb);
        for (int pos = 0; pos < 8 * kb; pos++)
            if (key_bit(k, kb, map, pos)) m[pos / 8] |= (uint8_t)(0x80 >> (pos % 8));
    }
    return 0;
}

/* --------------------------------------------------------------------------
 * Records.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint8_t *keys;
    uint8_t *vals;      /* may be NULL */
    int kb, vb, map, w;
    int64_t visits;     /* element placements done by the partition step */
    /* optional trace of every partition configuration (worked example) */
    int64_t *trace;
    int64_t trace_cap, trace_len;
    int64_t n;
} records;

static void exchange(records *r, int64_t i, int64_t j)
{
    uint8_t t[KB_MAX];
    if (i == j) return;
    memcpy(t, r->keys + i * r->kb, (size_t)r->kb);
    memcpy(r->keys + i * r->kb, r->keys + j * r->kb, (size_t)r->kb);
    memcpy(r->keys + j * r->kb, t, (size_t)r->kb);
    if (r->vals && r->vb > 0) {
        uint8_t u[16];
        memcpy(u, r->vals + i * r->vb, (size_t)r->vb);
        memcpy(r->vals + i * r->vb, r->vals + j * r->vb, (size_t)r->vb);
        memcpy(r->vals + j * r->vb, u, (size_t)r->vb);
    }
}

static int bit_of(const records *r, int64_t i, int pos)
{
    return key_bit(r->keys + i * r->kb, r->kb, r->map, pos);
}

/* One trace row: pos, lower, upper, lo, hi, then the first key byte of every
 * element (the worked example sorts 1-byte keys). */
static void trace_state(records *r, int pos, int64_t lower, int64_t upper,
                        int64_t lo, int64_t hi)
{
    if (!r->trace) return;
    int64_t row = 5 + r->n;
    if (r->trace_len + row > r->trace_cap) return;
    int64_t *t = r->trace + r->trace_len;
    t[0] = pos; t[1] = lower; t[2] = upper; t[3] = lo; t[4] = hi;
    for (int64_t i = 0; i < r->n; i++) t[5 + i] = r->keys[i * r->kb];
    r->trace_len += row;
}

/* --------------------------------------------------------------------------
 * Binar sort ("Operation of Algorithm"), run as iteration over a worklist of
 * pending sub-arrays ("Algorithm Variants": the recursion replaced by
 * iteration).  Each pending entry is one call of the method: a sub-array
 * [lower, upper] and the bit position to split it on.  For each entry the four
 * steps are taken in the paper's order:
 *   1. base case ("Evaluate for Recursive Base Case"): nothing to do when the
 *      bit positions are used up or the sub-array holds at most one element;
 *   2. bounds ("Initialize Starting Array Bounds"): the lower sub-array starts
 *      empty at `lower`, the upper sub-array starts empty above `upper`;
 *   3. partition ("Partition Array into Sub-arrays"): the working element is
 *      the first one not yet placed; its bit at `pos` is extracted; a zero
 *      extends the lower sub-array over it, a one exchanges it with the last
 *      unplaced element and extends the upper sub-array downwards over that
 *      slot; this repeats until no unplaced element is left;
 *   4. continuation ("Determine Recursive Call on Sub-arrays"): if either
 *      sub-array is empty the range passes through undivided to bit pos + 1;
 *      otherwise both sub-arrays are split on bit pos + 1, the lower one first.
 * The worklist is a stack, so the lower sub-array and everything below it is
 * finished before the upper one starts: the order of the recursive method.
 * The stack never holds more than w + 1 entries (at most one pending upper
 * sub-array per bit position, plus the entry being taken).
 * ------------------------------------------------------------------------ */
typedef struct { int64_t lower, upper; int pos; } pending;

static void binar(records *r, int64_t first, int64_t last, int pos0)
{
    pending *stack = malloc((size_t)(r->w + 2) * sizeof(pending));
    int top = 0;
    if (!stack) return;
    stack[top++] = (pending){first, last, pos0};
    while (top > 0) {
        const pending call = stack[--top];
        const int64_t lower = call.lower, upper = call.upper;
        const int pos = call.pos;

        /* step 1 */
        if (pos >= r->w || upper - lower < 1) continue;

        /* step 2: [lower, below) is the lower sub-array, [above, upper] the
         * upper one; the elements in [below, above) are not placed yet */
        int64_t below = lower, above = upper + 1;
        trace_state(r, pos, lower, upper, below, above - 1);

        /* step 3 */
        while (below < above) {
            r->visits++;
            if (bit_of(r, below, pos)) {
                above--;
                exchange(r, below, above);
            } else {
                below++;
            }
            trace_state(r, pos, lower, upper, below, above - 1);
        }

        /* step 4 (below == above: the split point) */
        if (below == lower || below == upper + 1) {
            stack[top++] = (pending){lower, upper, pos + 1};      /* pass-through */
        } else {
            stack[top++] = (pending){below, upper, pos + 1};      /* upper, taken second */
            stack[top++] = (pending){lower, below - 1, pos + 1};  /* lower, taken first */
        }
    }
    free(stack);
}

static int check_args(int64_t n, int kb, int map, int vb, int w)
{
    if (n < 0 || kb <= 0 || kb > KB_MAX || vb < 0 || vb > 16) return -1;
    if (map < 0 || map > 3) return -1;
    if (map == MAP_FLOAT && kb != 4 && kb != 8) return -1;
    if (w < 0 || w > 8 * kb) return -1;
    return 0;
}

/* Sorts each segment [offsets[s], offsets[s+1]) in place with binar sort on
 * bit positions 0 .. w-1.  Returns the number of element placements (the
 * quantity the time analysis bounds by w per element), or -1 on bad arguments. */
int64_t oracle_binar_sort(uint8_t *keys, uint8_t *vals, const int64_t *offsets,
                          int64_t num_segments, int kb, int map, int vb, int w)
{
    if (check_args(0, kb, map, vb, w) || num_segments < 0) return -1;
    records r = {keys, vals, kb, vb, map, w, 0, NULL, 0, 0, 0};
    for (int64_t s = 0; s < num_segments; s++) {
        if (offsets[s + 1] < offsets[s]) return -1;
        binar(&r, offsets[s], offsets[s + 1] - 1, 0);
    }
    return r.visits;
}

/* Binar sort of one array with every partition configuration recorded (rows
 * of 5 + n int64: pos, lower, upper, lo, hi, key bytes).  Returns the number of
 * int64 written, or -1. */
int64_t oracle_binar_sort_trace(uint8_t *keys, int64_t n, int kb, int map, int w,
                                int64_t *trace, int64_t trace_cap)
{
    if (check_args(n, kb, map, 0, w)) return -1;
    records r = {keys, NULL, kb, 0, map, w, 0, trace, trace_cap, 0, n};
    binar(&r, 0, n - 1, 0);
    return r.trace_len;
}

/* --------------------------------------------------------------------------
 * Parallel variant ("Algorithm Variants"): one counting pass groups the
 * elements by their leading b bits (processor p gets the elements whose leading
 * bits spell p); then every group is binar-sorted from bit b on, independently,
 * one thread per group.  Used only to time the oracle on all host cores.
 * ------------------------------------------------------------------------ */
typedef struct { records r; int64_t lower, upper; int pos; } group_job;

static void *group_worker(void *arg)
{
    group_job *g = (group_job *)arg;
    binar(&g->r, g->lower, g->upper, g->pos);
    return NULL;
}

int64_t oracle_binar_sort_parallel(uint8_t *keys, uint8_t *vals, int64_t n, int kb,
                                   int map, int vb, int w, int log2_groups)
{
    if (check_args(n, kb, map, vb, w) || log2_groups < 0 || log2_groups > 12) return -1;
    int b = log2_groups < w ? log2_groups : w;
    int64_t groups = (int64_t)1 << b;
    int64_t *count = calloc((size_t)groups + 1, sizeof(int64_t));
    uint8_t *tk = malloc((size_t)(n * kb + 1));
    uint8_t *tv = (vals && vb) ? malloc((size_t)(n * vb + 1)) : NULL;
    int64_t *gid = malloc((size_t)(n + 1) * sizeof(int64_t));
    group_job *jobs = calloc((size_t)groups, sizeof(group_job));
    pthread_t *th = calloc((size_t)groups, sizeof(pthread_t));
    if (!count || !tk || !gid || !jobs || !th || (vals && vb && !tv)) return -1;

    for (int64_t i = 0; i < n; i++) {
        int64_t g = 0;
        for (int p = 0; p < b; p++) g = 2 * g + key_bit(keys + i * kb, kb, map, p);
        gid[i] = g;
        count[g + 1]++;
    }
    for (int64_t g = 0; g < groups; g++) count[g + 1] += count[g];
    int64_t *next = calloc((size_t)groups, sizeof(int64_t));
    for (int64_t g = 0; g < groups; g++) next[g] = count[g];
    for (int64_t i = 0; i < n; i++) {
        int64_t d = next[gid[i]]++;
        memcpy(tk + d * kb, keys + i * kb, (size_t)kb);
        if (tv) memcpy(tv + d * vb, vals + i * vb, (size_t)vb);
    }
    memcpy(keys, tk, (size_t)(n * kb));
    if (tv) memcpy(vals, tv, (size_t)(n * vb));

    int64_t visits = n; /* the counting pass looks at every element once */
    for (int64_t g = 0; g < groups; g++) {
        records r = {keys, vals, kb, vb, map, w, 0, NULL, 0, 0, 0};
        jobs[g].r = r;
        jobs[g].lower = count[g];
        jobs[g].upper = count[g + 1] - 1;
        jobs[g].pos = b;
        pthread_create(&th[g], NULL, group_worker, &jobs[g]);
    }
    for (int64_t g = 0; g < groups; g++) {
        pthread_join(th[g], NULL);
        visits += jobs[g].r.visits;
    }
    free(count); free(next); free(tk); free(tv); free(gid); free(jobs); free(th);
    return visits;
}

/* --------------------------------------------------------------------------
 * Stable binary radix sort ("Sorting Formalism": among the permutations that
 * order the keys, the stable one keeps equal keys in their input order).
 * Least significant bit first, one bit per pass, each pass a stable split of
 * the segment into the elements whose bit is 0 followed by those whose bit is 1.
 * After the pass on bit 0 (the most significant) the segment is ordered by all
 * w bits, and equal keys are in input order because every pass kept it.
 * ------------------------------------------------------------------------ */
int oracle_stable_radix(uint8_t *keys, uint8_t *vals, const int64_t *offsets,
                        int64_t num_segments, int kb, int map, int vb, int w)
{
    if (check_args(0, kb, map, vb, w) || num_segments < 0) return -1;
    int64_t maxlen = 0;
    for (int64_t s = 0; s < num_segments; s++) {
        if (offsets[s + 1] < offsets[s]) return -1;
        if (offsets[s + 1] - offsets[s] > maxlen) maxlen = offsets[s + 1] - offsets[s];
    }
    uint8_t *tk = malloc((size_t)(maxlen * kb + 1));
    uint8_t *tv = malloc((size_t)(maxlen * (vb > 0 ? vb : 1) + 1));
    if (!tk || !tv) return -1;
    for (int64_t s = 0; s < num_segments; s++) {
        int64_t first = offsets[s], len = offsets[s + 1] - offsets[s];
        uint8_t *k = keys + first * kb;
        uint8_t *v = (vals && vb) ? vals + first * vb : NULL;
        for (int pos = w - 1; pos >= 0; pos--) {
            int64_t zeros = 0;
            for (int64_t i = 0; i < len; i++)
                if (key_bit(k + i * kb, kb, map, pos) == 0) zeros++;
            int64_t at0 = 0, at1 = zeros;
            for (int64_t i = 0; i < len; i++) {
                int64_t d = key_bit(k + i * kb, kb, map, pos) ? at1++ : at0++;
                memcpy(tk + d * kb, k + i * kb, (size_t)kb);
                if (v) memcpy(tv + d * vb, v + i * vb, (size_t)vb);
            }
            memcpy(k, tk, (size_t)(len * kb));
            if (v) memcpy(v, tv, (size_t)(len * vb));
        }
    }
    free(tk); free(tv);
    return 0;
}

/* --------------------------------------------------------------------------
 * One partition pass, k bits at a time: the records of [0, n) are split,
 * stably, into 2^k sub-arrays by the digit formed by bits pos .. pos+k-1 of
 * the encoding (bits past the end of the key read as 0).  Sub-array d is
 * written to [offsets[d], offsets[d+1]) of the output.  With k = 1 this is the
 * paper's lower/upper split with the input order kept inside each sub-array.
 * ------------------------------------------------------------------------ */
int oracle_partition_pass(const uint8_t *keys_in, const uint8_t *vals_in,
                          uint8_t *keys_out, uint8_t *vals_out, int64_t n,
                          int kb, int map, int vb, int pos, int k, int64_t *offsets)
{
    if (check_args(n, kb, map, vb, 8 * kb) || k < 1 || k > 16 || pos < 0 || pos >= 8 * kb)
        return -1;
    int64_t radix = (int64_t)1 << k;
    int64_t *digit = malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!digit) return -1;
    for (int64_t d = 0; d <= radix; d++) offsets[d] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t d = 0;
        for (int j = 0; j < k; j++) {
            int p = pos + j;
            int b = p < 8 * kb ? key_bit(keys_in + i * kb, kb, map, p) : 0;
            d = 2 * d + b;
        }
        digit[i] = d;
        offsets[d + 1]++;
    }
    for (int64_t d = 0; d < radix; d++) offsets[d + 1] += offsets[d];
    int64_t *next = malloc((size_t)radix * sizeof(int64_t));
    if (!next) { free(digit); return -1; }
    for (int64_t d = 0; d < radix; d++) next[d] = offsets[d];
    for (int64_t i = 0; i < n; i++) {
        int64_t at = next[digit[i]]++;
        memcpy(keys_out + at * kb, keys_in + i * kb, (size_t)kb);
        if (vals_in && vals_out && vb)
            memcpy(vals_out + at * vb, vals_in + i * vb, (size_t)vb);
    }
    free(digit); free(next);
    return 0;
}

/* --------------------------------------------------------------------------
 * Rank of one key by definition ("Sorting Formalism": in the sorted
 * permutation a key K sits after every key smaller than K): counts the input
 * keys whose encoding is below / not above that of `probe`.  With these, the
 * key at any output position i of a sort can be checked on its own:
 * less(K) <= i < less_or_equal(K).
 * ------------------------------------------------------------------------ */
static int compare_encoded(const uint8_t *a, const uint8_t *b, int kb, int map)
{
    for (int pos = 0; pos < 8 * kb; pos++) {
        int x = key_bit(a, kb, map, pos), y = key_bit(b, kb, map, pos);
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

int oracle_rank_of(const uint8_t *keys, int64_t n, int kb, int map, const uint8_t *probe,
                   int64_t *less, int64_t *less_or_equal)
{
    if (check_args(n, kb, map, 0, 8 * kb)) return -1;
    int64_t lt = 0, le = 0;
    for (int64_t i = 0; i < n; i++) {
        int c = compare_encoded(keys + i * kb, probe, kb, map);
        if (c < 0) lt++;
        if (c <= 0) le++;
    }
    *less = lt;
    *less_or_equal = le;
    return 0;
}

/* Index of the j-th (0-based) input key equal to `probe`, or -1: in the stable
 * order the j-th copy of a key in the output is the j-th copy in the input. */
int64_t oracle_occurrence(const uint8_t *keys, int64_t n, int kb, const uint8_t *probe, int64_t j)
{
    for (int64_t i = 0; i < n; i++) {
        if (memcmp(keys + i * kb, probe, (size_t)kb) == 0) {
            if (j == 0) return i;
            j--;
        }
    }
    return -1;
}

/* --------------------------------------------------------------------------
 * Byte strings of different lengths ("The Other Universal Property": strings
 * are sorted by their encoding; "Recursion Analysis": a string costs its
 * average length in bit passes).  The paper gives no rule for strings of
 * unequal length; the order used is the plain lexicographic one: the first
 * differing byte decides (unsigned), and a string that is a proper prefix of
 * another sorts first.  Equal strings keep their input order (the stable
 * permutation of "Sorting Formalism").
 *
 * oracle_sort_strings writes order[k] = index of the k-th string in that
 * order, string i being bytes[offsets[i] .. offsets[i+1]).  It is the plain
 * definition: a merge sort of the indices (stable: on a tie the left run's
 * element is taken first) with the comparison written out byte by byte.
 * ------------------------------------------------------------------------ */
static int compare_strings(const uint8_t *bytes, const int64_t *offsets, uint32_t a, uint32_t b)
{
    const int64_t la = offsets[a + 1] - offsets[a], lb = offsets[b + 1] - offsets[b];
    const uint8_t *sa = bytes + offsets[a], *sb = bytes + offsets[b];
    const int64_t common = la < lb ? la : lb;
    for (int64_t i = 0; i < common; i++)
        if (sa[i] != sb[i]) return sa[i] < sb[i] ? -1 : 1;
    if (la != lb) return la < lb ? -1 : 1;
    return 0;
}

int oracle_sort_strings(const uint8_t *bytes, const int64_t *offsets, int64_t n, uint32_t *order)
{
    if (n < 0 || n > 0xFFFFFFFFLL) return -1;
    for (int64_t i = 0; i < n; i++)
        if (offsets[i + 1] < offsets[i] || offsets[i] < 0) return -1;
    uint32_t *tmp = malloc((size_t)(n + 1) * sizeof(uint32_t));
    if (!tmp) return -1;
    for (int64_t i = 0; i < n; i++) order[i] = (uint32_t)i;
    /* bottom-up merge sort: runs of width 1, 2, 4, ... */
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi)
                tmp[k++] = compare_strings(bytes, offsets, order[j], order[i]) < 0 ? order[j++]
                                                                                   : order[i++];
            while (i < mid) tmp[k++] = order[i++];
            while (j < hi) tmp[k++] = order[j++];
        }
        memcpy(order, tmp, (size_t)n * sizeof(uint32_t));
    }
    free(tmp);
    return 0;
}
