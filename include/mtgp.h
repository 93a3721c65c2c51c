/*
 * libmtgp -- MTGP generation on one GB300 GPU (sm_103a), C ABI.
 *
 * MTGP is the Mersenne Twister for Graphic Processors of Saito and Matsumoto
 * ("Variants of Mersenne Twister Suitable for Graphic Processors", arXiv
 * 1005.4973).  One generator's state of N = ceil(mexp / 32) 32-bit words is
 * owned by one thread block, which computes many steps of the F2-linear
 * recursion at once (Sec. 3.2), tempers them (Sec. 3.7) and writes uint32 or
 * single-precision outputs (Sec. 6) to device memory.
 *
 * Conventions for every call:
 *   - Functions return an mtgp_status and never abort; on failure
 *     mtgp_last_error() returns a message for the calling thread.
 *   - Pointers named dev_* are raw CUDA device pointers owned by the caller.
 *     Pointers named host_* are host pointers owned by the caller.
 *   - stream arguments are cudaStream_t values passed as void * (NULL is the
 *     legacy default stream).  Calls are stream-ordered and asynchronous
 *     unless stated otherwise; nothing synchronises implicitly.
 *   - Objects (mtgp_state, mtgp_pool) are created and owned by the library;
 *     the caller destroys them.  Their generator states stay resident in
 *     device memory between calls, so generation continues where the last
 *     call stopped (Sec. 8).
 *   - A pool is used by at most one stream at a time: a call on a second
 *     stream while work from the first is still in flight returns MTGP_EBUSY.
 */
#ifndef MTGP_H
#define MTGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MTGP_MAX_N 4096u          /* largest state, in 32-bit words             */
#define MTGP_PARAMS_VERSION 1u

typedef enum mtgp_status {
    MTGP_OK = 0,
    MTGP_EINVAL = 1,     /* an argument is out of range or inconsistent        */
    MTGP_ENOMEM = 2,     /* device or host allocation failed                    */
    MTGP_ECUDA = 3,      /* a CUDA runtime call failed (message has the code)   */
    MTGP_ETIMEOUT = 4,   /* a bounded device-side wait ran out                  */
    MTGP_EBUSY = 5       /* the object has work in flight on another stream     */
} mtgp_status;

/* Output types (Sec. 6).  Every output occupies 4 bytes. */
typedef enum mtgp_dtype {
    MTGP_U32 = 0,        /* tempered 32-bit integer o_{N+i}                      */
    MTGP_F32_12 = 1,     /* float in [1,2): 0x3F800000 | (o >> 9)                */
    MTGP_F32_01 = 2      /* float in [0,1): the [1,2) float minus 1.0f (exact)  */
} mtgp_dtype;

typedef enum mtgp_layout {
    MTGP_LAYOUT_BLOCKED = 0,      /* request j writes its n numbers contiguously
                                     from element out_offset                      */
    MTGP_LAYOUT_INTERLEAVED = 1   /* all requests have the same n; numbers go out
                                     in chunks of `chunk` per request, round robin
                                     over the requests in array order             */
} mtgp_layout;

/*
 * One MTGP parameter set: the recursion parameters (N, M = pos, w = 32, r,
 * sh1, sh2, R) of the Definition in Sec. 3.6 and the tempering parameter T of
 * the Definition in Sec. 3.7, with R and T given as their 16-entry look-up
 * tables: rec_tbl[b] = b R and tmp_tbl[b] = b T for the 4-bit row vector b
 * (Sec. 3.6, 3.7).  N = ceil(mexp / 32), r = 32 N - mexp (Sec. 3.3),
 * mask = BITMASK(32, r): the 32 - r MSBs set (Sec. 3.6).  `id` is the 32-bit
 * generator ID of Sec. 5 (informational; it is embedded in R by the drawer).
 * The single-precision table of Sec. 6 is derived from tmp_tbl.
 */
typedef struct mtgp_params {
    uint32_t mexp, N, r, mask, pos, sh1, sh2, id;
    uint32_t rec_tbl[16];
    uint32_t tmp_tbl[16];
} mtgp_params;

typedef struct mtgp_state mtgp_state;   /* one device-resident generator       */
typedef struct mtgp_pool mtgp_pool;     /* many device-resident generators     */

/* One unit of batched work: n numbers of generator `gen` (an index into the
 * pool, 0 .. count-1) of type dtype.  Requests naming the same generator in
 * one call are applied in array order, each continuing the stream. */
typedef struct mtgp_request {
    uint32_t gen;
    uint32_t dtype;          /* mtgp_dtype                                       */
    uint64_t n;              /* numbers to generate; 0 is allowed (no-op)       */
    uint64_t out_offset;     /* element offset into the output (blocked layout) */
} mtgp_request;

/* Launch configuration of a pool (chosen by mtgp_autotune or set by hand).
 * A generator runs in rounds of S = N - M words (Sec. 3.2).  Plain form: each
 * of the `threads` threads owns ceil(S / threads) of the S columns and also
 * tempers and stores them.  Split form: the first half of the block runs the
 * recursion (owning ceil(S / (threads / 2)) columns each) and the second half
 * tempers, converts and stores finished rounds.  Wide form: each thread owns
 * groups of 4 adjacent columns, whose reads overlap (x_{i+1} of one column is
 * x_i of the next) and whose outputs leave in one 16-byte store; blocked
 * layouts only (interleaved calls run in the plain form).  Pair form: each
 * thread owns two adjacent columns per slot (x_{i+1} and one tempering word
 * shared within the pair, 8-byte stores), 128 threads.  Dual form: a block of
 * 128 threads runs two work items at once, a round of each between block
 * barriers, each in its own half of the shared buffer; every generator of a
 * launch must have 257 <= S <= 384 (MTGP 11213), or the launch fails with
 * MTGP_EINVAL.  mtgp_autotune tries every form. */
typedef struct mtgp_config {
    uint32_t threads;          /* threads per block: plain 32, 64, 128, 256, 512
                                  (at most 11, 12, 11, 6, 8 columns per thread);
                                  split 128, 256, 512, 1024 (at most 12, 11, 6, 3);
                                  flow 128, 256, 512, 1024 (at most 12, 11, 6, 8);
                                  wide 96, 128, 192 (rounds of at most 1529 words);
                                  pairs 128 (at most 6 pairs); dual 128 (3).  Plain
                                  form: a launch whose rounds need more columns
                                  than this size has a kernel for runs with the
                                  smallest larger size that has one (256, 512)    */
    uint32_t persistent;       /* 1 (default): grid of SMs x blocks_per_sm blocks
                                  taking work items longest first from a device
                                  counter; 0: one block per work item               */
    uint32_t blocks_per_sm;    /* persistent grid occupancy; 0 = what the kernel's
                                  registers allow, shared buffers sized for it, and
                                  a launch whose items all fit at once runs one
                                  block per item                                    */
    uint32_t chunk;            /* interleaved layout chunk, power of two >= 32       */
    uint32_t buffer_words;     /* shared-memory words per block, 0 = sized from the
                                  launch (>= 2N + owners ceil(S / owners) + 32 is
                                  required, owners = threads or threads / 2, twice
                                  that for the dual form's two halves; wide
                                  form: 4 floor(buffer_words / 4) >= 2N + S + 24)    */
    uint32_t form;             /* 0 plain, 1 split (recursion and output warp groups
                                  handing rounds over through named barriers),
                                  2 flow (split groups, and each recursion warp
                                  waits only for the warps holding its inputs),
                                  3 wide (4 adjacent columns per thread),
                                  4 pairs (2 adjacent columns per thread),
                                  5 dual (two items per block; always pulls
                                  items from the work counter)                      */
    uint32_t pieces;           /* jump-ahead (Sec. 7): a generator's work in one call
                                  (blocked layout) may run as up to this many pieces
                                  on separate blocks, piece m starting from the state
                                  m L numbers ahead, computed on the GPU before the
                                  launch; outputs are identical.  0 = auto (about 16
                                  blocks per SM; up to 64 per generator), 1 = never
                                  split, else at most 256                           */
    uint32_t piece_log2;       /* pieces hold at least 2^piece_log2 numbers; 0 = 20,
                                  else 10 .. 40                                    */
    uint32_t round_words;      /* words per round (Sec. 3.2: any n <= S = N - M
                                  consecutive words are independent): 0 = S; the
                                  wide form takes rounds of min(S, round_words),
                                  a multiple of 4 >= 8; the other forms keep the
                                  round's column slots in registers from round to
                                  round, which needs rounds of exactly S words     */
} mtgp_config;

/* ---- library ------------------------------------------------------------ */

/* Version string of the library. */
const char *mtgp_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *mtgp_last_error(void);

/* ---- parameter sets (host only, pure) ------------------------------------ */

/*
 * Draws a synthetic parameter set of exponent mexp with the structure that
 * MTGPDC gives its sets (Sec. 5): ID[31:16] in the 16 MSBs of row 0 of R,
 * ID[15:0] in MSB positions 13..28 of row 1, the LSB nibbles of the rows
 * redrawn until the 4x4 block plus the identity is invertible, the rest of R
 * and all of T random, sh1 = 13, sh2 = 4, M uniform in 2 < M < N - [N]_2
 * (the Sec. 3.5 range M >= 2, N - M >= [N-2]_2 where that one is empty).
 * Randomness: the SplitMix64 stream started at param_seed, drawn in the order
 * M, rows of R, rejected LSB nibbles, rows of T.  Drawn sets are not searched
 * for full period.  Errors: MTGP_EINVAL if mexp < 65 or N > MTGP_MAX_N or
 * out is NULL.
 */
mtgp_status mtgp_params_draw(uint32_t mexp, uint64_t param_seed, uint32_t id, mtgp_params *out);

/*
 * Checks a parameter set: N, r and mask consistent with mexp (Sec. 3.3, 3.6),
 * 2 <= pos < N, 1 <= sh1, sh2 <= 31, both tables F2-linear (tbl[a ^ b] =
 * tbl[a] ^ tbl[b], so tbl[0] = 0), the LSB block of R invertible (Sec. 5), and
 * N <= MTGP_MAX_N.  Returns MTGP_OK or MTGP_EINVAL with the reason.
 */
mtgp_status mtgp_params_validate(const mtgp_params *p);

/*
 * Recursion-parameter search of MTGPDC (Sec. 5) on the host cores: candidates
 * t = 0, 1, ... are mtgp_params_draw(mexp, seed0 + t, id) (ID embedded in R,
 * R4 + I invertible, sh1 = 13, sh2 = 4, M in Sec. 5's range).  A candidate is
 * accepted when the Berlekamp-Massey polynomial of the MSB sequence of 2 mexp
 * words of its recursion (from a SplitMix64-filled state) has degree mexp and
 * is irreducible -- then it is the characteristic polynomial of the
 * transition F and primitive (mexp a Mersenne exponent), so the period is
 * 2^mexp - 1 (Sec. 3.3).  Irreducibility: x^(2^mexp) = x mod phi and no root
 * in F2, with an early gcd against prod_{k <= 40} (x^(2^k) - x).  Returns the
 * smallest accepted t (whatever the thread count): the set in *out, seed0 + t
 * in *found_seed, t + 1 in *tries, and, if charpoly is not NULL, phi (bit j of
 * word j/64 = coefficient of x^j; charpoly_words >= mexp / 64 + 1).
 * threads = 0 uses every host core.  MTGP_EINVAL if none of max_tries
 * candidates qualifies.  The tempering table of the result is the drawn one;
 * mtgp_params_temper_search replaces it by the search of Sec. 5.  For mexp
 * 11213 (seed0 1, 14229 candidates) about 24 s of 16 cores; the cost grows
 * roughly as mexp^3.  mtgp_params_search_gpu gives the same result faster.
 */
mtgp_status mtgp_params_search(uint32_t mexp, uint64_t seed0, uint32_t id, uint64_t max_tries, uint32_t threads,
                               mtgp_params *out, uint64_t *found_seed, uint64_t *tries, uint64_t *charpoly,
                               uint32_t charpoly_words);

/*
 * The same search (same candidates, same acceptance, same result) with the
 * polynomial work on the GPU: candidates run in batches of up to 4096; the
 * host cores draw them and walk their MSB sequences, one warp per candidate
 * finds the sequence's minimal polynomial on `stream`, and one block per
 * candidate of degree mexp tests it for irreducibility (the test of
 * mtgp_f2_irreducible_gpu; the survivors of its sieve are squared on streams
 * of the call's own while later batches run, and batches are settled in
 * order).  mexp > 32.  Allocates and frees its device buffers and streams
 * (about 4 x 4096 x mexp / 8 bytes); synchronous.  Errors as
 * mtgp_params_search, plus MTGP_ECUDA.
 */
mtgp_status mtgp_params_search_gpu(uint32_t mexp, uint64_t seed0, uint32_t id, uint64_t max_tries,
                                   uint32_t threads, void *stream, mtgp_params *out, uint64_t *found_seed,
                                   uint64_t *tries, uint64_t *charpoly, uint32_t charpoly_words);

/*
 * Dimensions of equidistribution (Sec. 3.4, 3.8; Table 1): k(v) for v = 1 ..
 * 32 of the tempered uint32 output -- the largest k such that the v most
 * significant bits of k consecutive outputs are equidistributed over a
 * period -- to kv[v - 1], and the total dimension defect sum_v (floor(mexp /
 * v) - k(v)) to *delta (if not NULL).  For a full-period set (characteristic
 * polynomial P of degree mexp, irreducible) k(v) is the least max-degree of
 * the nonzero vectors (f_1 .. f_v) over F2[t] with sum_j f_j h_j = 0 mod P,
 * h_j / P the generating function of output bit 32 - j: a lattice that the
 * library reduces to weak Popov form, one bit at a time (Sec. 5 uses a
 * lattice method too); a fraction of a second for mexp 11213.  Other sets
 * (P of lower degree: k(v) then describes the orbit of one state) fall back
 * to row reduction of the states F^j s, one host thread per v (seconds).
 */
mtgp_status mtgp_params_equidistribution(const mtgp_params *p, uint32_t threads, uint32_t *kv, uint32_t *delta);

/* The same for the v LEAST significant bits (k'(v) of Sec. 5: bits 0 .. v-1). */
mtgp_status mtgp_params_equidistribution_lsb(const mtgp_params *p, uint32_t threads, uint32_t *kv,
                                             uint32_t *delta);

/*
 * Tempering search of Sec. 5 for a full-period set *in (its tmp_tbl is
 * ignored): the four tempering rows start at zero; for row 0, 1, 2, 3 in
 * turn, the 23 MSBs are set in windows of bits j .. e-1 counted from the MSB
 * (j = 0, 5, 10, 15, 20; e = min(j + 5, 23)), each to the pattern with the
 * least d(1) + .. + d(e) (every pattern of the window tried, the smallest
 * pattern value on ties); then, row by row, the 9 LSBs in windows of bits
 * j .. e-1 counted from the LSB (j = 0, 5; e = min(j + 5, 9)) against the
 * defects d'(1) + .. + d'(e) of the v least significant bits.  *out = *in
 * with the table of the rows found (bit 3 of the index selects row 0), its
 * total MSB defect to *delta (if not NULL).  threads = 0 uses every host
 * core (the patterns of a window run in parallel).  MTGP_EINVAL for a set
 * that is not of full period.
 */
mtgp_status mtgp_params_temper_search(const mtgp_params *in, uint32_t threads, mtgp_params *out, uint32_t *delta);

/*
 * Table 1 style report of a set (Sec. 3.8): one line per v = 1 .. 32 with
 * v, k(v), d(v) = floor(mexp / v) - k(v) and r(v) = 100 d(v) / (k(v) + d(v))
 * in percent, then "total dimension defect <sum of d(v)>".  NUL-terminated
 * text into buf (len bytes; MTGP_EINVAL if too small, 2 KiB suffice).
 */
mtgp_status mtgp_params_report(const mtgp_params *p, uint32_t threads, char *buf, size_t len);

/*
 * MTGPDC record of a searched set (Sec. 5): comma-separated mexp, N, pos,
 * sh1, sh2, id, the 16 rec_tbl and 16 tmp_tbl entries (8 hexadecimal
 * digits each), the SHA-1 digest of the characteristic polynomial (of its
 * coefficients written as '0' / '1' characters from x^0 up to x^mexp), its
 * number of nonzero terms, and the total dimension defect.  charpoly: bit i
 * of word i / 64 = coefficient of x^i (as mtgp_params_search returns it).
 */
mtgp_status mtgp_params_record(const mtgp_params *p, const uint64_t *charpoly, uint32_t charpoly_words,
                               uint32_t threads, char *buf, size_t len);

/* ---- single generator (Sec. 8 host/kernel flow) --------------------------- */

/*
 * Creates one generator with parameter set p, generator ID gen_id and 64-bit
 * seed, and initialises its state in device memory on `stream` (the paper
 * leaves seeding open; the state words are SplitMix64 outputs keyed by seed
 * and gen_id, with the all-zero state excluded).  The library owns the state.
 * Errors: MTGP_EINVAL (invalid p), MTGP_ENOMEM, MTGP_ECUDA.
 */
mtgp_status mtgp_state_create(const mtgp_params *p, uint32_t gen_id, uint64_t seed,
                              void *stream, mtgp_state **out);

/*
 * Generates the next n numbers of the generator as dtype into dev_out
 * (>= 4 n bytes, 4-byte aligned, caller-owned) and advances its state by n,
 * stream-ordered on `stream`: one block loads the state into a shared-memory
 * ring, runs rounds of the recursion (Sec. 3.2, 3.6), tempers (Sec. 3.7),
 * converts (Sec. 6), stores, and writes the state back (Sec. 8).  n = 0 is a
 * no-op.  Errors: MTGP_EINVAL (bad dtype, NULL dev_out with n > 0),
 * MTGP_EBUSY, MTGP_ECUDA.
 */
mtgp_status mtgp_generate(mtgp_state *s, mtgp_dtype dt, void *dev_out, uint64_t n, void *stream);

/*
 * Checkpoint: copies the generator (parameters, stream position, state) to
 * host_buf.  If host_buf is NULL, only *bytes is set to the size needed.
 * Synchronises with the last stream the generator was used on.
 */
mtgp_status mtgp_state_save(const mtgp_state *s, void *host_buf, size_t *bytes);

/* Restores a checkpoint made by mtgp_state_save (same N).  Synchronous. */
mtgp_status mtgp_state_load(mtgp_state *s, const void *host_buf, size_t bytes);

/* Numbers generated so far by the generator (its stream position). */
mtgp_status mtgp_state_position(const mtgp_state *s, uint64_t *pos);

/* Frees the generator (after synchronising with its last stream). */
void mtgp_state_destroy(mtgp_state *s);

/* ---- many generators: batched and served forms ---------------------------- */

/*
 * Creates `count` device-resident generators: generator i has parameter set
 * ps[i], ID gen_ids[i] and seed seeds[i] (the same seeding as
 * mtgp_state_create).  Parameter sets may mix exponents.  States are laid out
 * back to back in one device buffer, each 16-byte aligned.
 * Errors: MTGP_EINVAL, MTGP_ENOMEM, MTGP_ECUDA.
 */
mtgp_status mtgp_pool_create(const mtgp_params *ps, const uint32_t *gen_ids, const uint64_t *seeds,
                             uint32_t count, void *stream, mtgp_pool **out);

/* Number of generators and device bytes held by the pool. */
mtgp_status mtgp_pool_info(const mtgp_pool *p, uint32_t *count, uint64_t *device_bytes);

/* Reads / sets the pool's launch configuration (validated: MTGP_EINVAL). */
mtgp_status mtgp_pool_get_config(const mtgp_pool *p, mtgp_config *cfg);
mtgp_status mtgp_pool_set_config(mtgp_pool *p, const mtgp_config *cfg);

/*
 * Runs nreq requests in one generation launch on `stream`.  Requests of the
 * same generator are grouped, in array order, into one work item (a
 * generator's stream is sequential, Sec. 3.2); work items of different
 * generators run in parallel blocks.  In the blocked layout an item may run as
 * jump-ahead pieces (mtgp_config.pieces), whose start states one jump launch
 * computes first; the outputs are the same.  Blocked layout:
 * request j writes elements [out_offset, out_offset + n) of dev_out.
 * Interleaved layout: every request has the same n and a distinct generator,
 * out_offset is ignored, and number k of request j goes to element
 * (k / chunk) * (nreq * chunk) + j * chunk + k % chunk.
 * dev_out must be 4-byte aligned (16-byte aligned for the fastest stores) and
 * large enough; it is caller-owned.  A stream being captured into a CUDA
 * graph is refused, as by every pool call that takes a stream: the work list
 * is copied from a pool buffer that the next call reuses (mtgp_graph_create
 * captures a pool launch).  Errors: MTGP_EINVAL (bad index, dtype or layout,
 * stream under capture), MTGP_EBUSY, MTGP_ENOMEM, MTGP_ECUDA.
 */
mtgp_status mtgp_pool_generate(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq,
                               void *dev_out, mtgp_layout layout, void *stream);

/*
 * End-to-end form of mtgp_pool_generate: the outputs land in HOST memory.
 * Generation runs into library-owned device staging buffers of at most
 * staging_bytes each (0 = 1 GiB) and each slice is copied to host_out while
 * the next one is generated.  host_out should be pinned (cudaHostAlloc) for
 * full copy bandwidth.  Returns after all copies completed (synchronous).
 */
mtgp_status mtgp_pool_generate_host(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq,
                                    void *host_out, mtgp_layout layout, uint64_t staging_bytes,
                                    void *stream);

/* Stream position of generator i (numbers generated so far). Synchronous. */
mtgp_status mtgp_pool_position(mtgp_pool *p, uint32_t i, uint64_t *pos);

/*
 * Copies generator i's state words (N of them, oldest first: x_k .. x_{k+N-1}
 * after k numbers) to host_state.  Synchronous.  For tests and checkpoints.
 */
mtgp_status mtgp_pool_read_state(mtgp_pool *p, uint32_t i, uint32_t *host_state);

/* Checkpoint of the whole pool: same contract as mtgp_state_save / _load. */
mtgp_status mtgp_pool_save(mtgp_pool *p, void *host_buf, size_t *bytes);
mtgp_status mtgp_pool_load(mtgp_pool *p, const void *host_buf, size_t bytes);

/* Frees the pool (after synchronising with its last stream). */
void mtgp_pool_destroy(mtgp_pool *p);

/*
 * The project's autotuner: picks the launch configuration and the output
 * layout for these requests by timing candidates on `stream`, the requests
 * written to dev_scratch (caller-owned, 4 sum(n) bytes).  Stage 1 tries every
 * form (plain, split, flow, wide, pairs) with its block sizes, words per round
 * (mtgp_config.round_words: S, 128 or 256 for the wide form), persistent grids
 * of 0 / 2 / 4 / 8 blocks per SM or one block per item, and jump-ahead pieces
 * (auto or none), in the blocked layout when `layouts` allows it (bit 0;
 * else interleaved).  Stage 2, when `layouts` bit 1 allows the interleaved
 * layout and the requests qualify (equal lengths, distinct generators),
 * tries it with chunks of 2^8, 2^12 and 2^16 numbers (those dividing the
 * length) for the best configuration of stage 1.  The generators' states are
 * saved before and restored after, so tuning does not advance any stream (the
 * restore empties the work lists of the pool's graphs that hold jump-ahead
 * pieces, as mtgp_pool_load does).  On success the best configuration is set
 * on the pool and copied to *best, the layout to *best_layout and its time to
 * *best_ms (each if not NULL).  Synchronous.
 */
mtgp_status mtgp_autotune(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq, void *dev_scratch,
                          uint32_t layouts, void *stream, mtgp_config *best, mtgp_layout *best_layout,
                          float *best_ms);

/*
 * Error word of the pool's last launches: bit 0 a generator did not fit the
 * launch's kernel shape or shared buffer, bit 1 a bounded wait between warps
 * ran out (flow form).  Synchronous; clears the word.  Outputs of a launch
 * that set a bit are invalid.
 */
mtgp_status mtgp_pool_errors(mtgp_pool *p, uint32_t *flags);

/* Kernels launched so far by the pool's generation calls (generation, plus
 * the two jump-ahead kernels of calls that split work into pieces). */
mtgp_status mtgp_pool_launch_count(const mtgp_pool *p, uint64_t *launches);

/*
 * Flow form (mtgp_config.form = 2): polls per bounded wait between warps in
 * its later launches (0, the default: 2^22).  A wait that runs out sets bit 1
 * of the error word (mtgp_pool_errors), the warp stops waiting, the launch
 * ends and its outputs are invalid; the context stays usable.  Graphs capture
 * the limit in force when they are created.  Waits for queued work.
 */
mtgp_status mtgp_pool_set_spin_limit(mtgp_pool *p, uint32_t polls);

/*
 * Per-kernel timing, for measurement.  With entries > 0, each later
 * mtgp_pool_generate call that launches work records three CUDA events on its
 * stream: before its jump-ahead launch (Sec. 7), and before and after its
 * generation launch, into a ring of `entries` records (created here, so that
 * the timed calls create nothing).  entries = 0 turns it off.  Waits for the
 * pool's queued work.
 */
mtgp_status mtgp_pool_set_timing(mtgp_pool *p, uint32_t entries);

/*
 * The device durations, in ms, of the last `count` recorded calls (oldest
 * first): jump_ms[k] the jump-ahead launch (0 if the call had none), gen_ms[k]
 * the generation launch.  Waits for those calls.  MTGP_EINVAL if fewer were
 * recorded.
 */
mtgp_status mtgp_pool_kernel_times(mtgp_pool *p, uint32_t count, float *jump_ms, float *gen_ms);

/* ---- jump-ahead (Sec. 7) ------------------------------------------------------
 *
 * Sec. 7 observes that one generator's stream can be produced by several
 * processors if the state n outputs ahead can be computed without producing
 * them.  For a state s of the linear transition F (Sec. 3.3) the library finds
 * an annihilating polynomial psi, psi(F) s = 0: the Berlekamp-Massey minimal
 * polynomial of a bit sequence read off the walk from s (a linear functional
 * of the state), checked on the GPU by computing phi(F) s and repeated on the
 * remainder until it vanishes.  Then F^J s = g(F) s with g = x^J mod psi, an
 * XOR of the states F^i s that g's coefficients select.  psi of a state also
 * annihilates every later state, so it is computed once per generator (and
 * again after mtgp_pool_load).  The pool uses this to split long requests
 * into pieces (mtgp_config.pieces); the calls below expose it directly.
 */

/* Advances generator i by `steps` outputs without producing them: state and
 * position become exactly those after generating `steps` numbers.  The first
 * use for a generator computes psi (GPU walk plus host Berlekamp-Massey:
 * milliseconds for mexp 11213, about a second for 44497); each jump then
 * costs O(log steps) polynomial squarings modulo psi on the host and one
 * O(mexp N) GPU pass.  Synchronous. */
mtgp_status mtgp_pool_jump(mtgp_pool *p, uint32_t i, uint64_t steps, void *stream);
mtgp_status mtgp_state_jump(mtgp_state *s, uint64_t steps, void *stream);

/* psi of generator i's current stream (computed if not known yet): its degree
 * (<= mexp) goes to *degree and its coefficients to poly (bit j of word j/64 =
 * coefficient of x^j) if poly_words >= degree / 64 + 1; with poly NULL only
 * the degree is returned.  MTGP_EINVAL if poly is too small.  Synchronous. */
mtgp_status mtgp_pool_annihilator(mtgp_pool *p, uint32_t i, uint64_t *poly, uint32_t poly_words,
                                  uint32_t *degree, void *stream);

/* F2[x] routines behind jump-ahead (host only, pure).  A polynomial is a
 * little-endian array of 64-bit words: bit j of word j/64 is the coefficient
 * of x^j.  *deg receives the result's degree (-1 for zero).  MTGP_EINVAL if a
 * pointer is NULL, the modulus has degree < 1, or out has fewer than
 * deg / 64 + 1 words (then *deg still holds the degree).
 *   minpoly:  minimal polynomial of the bit sequence bits[0 .. n) (bit i of
 *             bits[i/64]) in annihilator form, sum_j c_j s_{k+j} = 0 for all k
 *             (Berlekamp-Massey; exact when the linear complexity <= n/2)
 *   mulmod:   a b mod m
 *   xpow_mod: x^e mod m */
mtgp_status mtgp_f2_minpoly(const uint64_t *bits, uint64_t n, uint64_t *out, uint32_t out_words, int64_t *deg);
/* Irreducibility over F2 on the GPU of `count` polynomials (host memory,
 * `words` 64-bit words each in the layout above), the acceptance test of the
 * Sec. 5 recursion search: verdicts[j] = 1 if polynomial j has degree exactly
 * p and is irreducible, else 0.  p must be a prime > 32 (the test is
 * Rabin's for prime degree: no root in F2 and x^(2^p) = x mod phi, after a
 * gcd against the product of x^(2^k) - x for 20 < k <= 40 that rejects
 * polynomials with a factor of degree <= 40); words >= p / 64 + 1.  One
 * block per polynomial on `stream`; synchronous; the device buffers are
 * allocated and freed by the call.  MTGP_EINVAL for NULL pointers, count 0,
 * p not prime or too small, or too few words; MTGP_ENOMEM; MTGP_ECUDA. */
mtgp_status mtgp_f2_irreducible_gpu(const uint64_t *polys, uint32_t count, uint32_t words, uint32_t p,
                                    void *stream, uint8_t *verdicts);
mtgp_status mtgp_f2_mulmod(const uint64_t *a, uint32_t a_words, const uint64_t *b, uint32_t b_words,
                           const uint64_t *m, uint32_t m_words, uint64_t *out, uint32_t out_words, int64_t *deg);
mtgp_status mtgp_f2_xpow_mod(uint64_t e, const uint64_t *m, uint32_t m_words, uint64_t *out, uint32_t out_words,
                             int64_t *deg);

/* ---- graph-captured batched launch --------------------------------------------
 *
 * Batching across many generators (not in the paper, which launches once per
 * call, Sec. 8): one persistent launch -- a grid of SMs x blocks_per_sm blocks
 * pulling work items longest first -- is captured once into a CUDA graph whose
 * work list, work-item count and output base live in a library-owned device
 * buffer.  Each mtgp_graph_set_requests rewrites that buffer (one async copy
 * on `stream`) and each mtgp_graph_launch replays the graph, so the launch
 * cost stays constant however the requests change.
 */
typedef struct mtgp_graph mtgp_graph;

/* Captures the launch for pool p with the pool's configuration (persistent),
 * sized for every generator of the pool and at most max_items work items
 * and max_items segments per replay.  Unless the pool's configuration has
 * pieces = 1, the capture also holds a jump launch (Sec. 7) before the
 * generation launch, and the graph owns device room for max_items piece
 * states (max_items x N words): long requests then run as jump-ahead pieces,
 * each replay computing their start states from the generators' current
 * states.  mtgp_pool_load, and any call on the pool that has to evict cached
 * jump polynomials (more than 1 GiB of them), empty the work lists of the
 * pool's graphs that hold pieces: their replays generate nothing until the
 * next mtgp_graph_set_requests.  Destroy a pool's graphs before the pool.
 * Synchronous.  Errors: MTGP_EINVAL, MTGP_ENOMEM, MTGP_ECUDA. */
mtgp_status mtgp_graph_create(mtgp_pool *p, uint32_t max_items, void *stream, mtgp_graph **out);

/* Sets the requests of the next replays: same contract as mtgp_pool_generate
 * (grouping, order, layouts, dev_out), stream-ordered on `stream`.  The work
 * list stays in place for later replays until the next call.  Pieces are
 * planned as for mtgp_pool_generate when they fit the graph's max_items and
 * piece-state room, else the requests run as whole work items.  On an error
 * the graph's work list is emptied (replays then generate nothing). */
mtgp_status mtgp_graph_set_requests(mtgp_graph *g, const mtgp_request *reqs, uint32_t nreq, void *dev_out,
                                    mtgp_layout layout, void *stream);

/* Replays the captured launch on `stream`: generates the current requests,
 * each replay continuing the generators' streams. */
mtgp_status mtgp_graph_launch(mtgp_graph *g, void *stream);

/* Error word of the graph's launches (as mtgp_pool_errors).  Synchronous. */
mtgp_status mtgp_graph_errors(mtgp_graph *g, uint32_t *flags);

/* Frees the graph (after the pool's work finished). */
void mtgp_graph_destroy(mtgp_graph *g);

/* ---- continuous-batching server ----------------------------------------------
 *
 * Serving loop over a pool (not in the paper): requests (generator, dtype, n)
 * arrive at any time; each mtgp_server_poll retires finished ticks, admits
 * pending requests in submission order while a slot is free and the output
 * fits in the server's device arena (admission by free memory), and launches
 * one tick -- one replay of the pool's captured persistent launch
 * (mtgp_graph_*) that advances every admitted request by up to `chunk`
 * numbers.  Requests that arrive while others are on the GPU join at the next
 * tick.  A generator's stream is sequential (Sec. 3.2), so its requests are
 * served one after another in submission order; requests of different
 * generators run in the same ticks.  Every result equals what the same
 * generator's requests give alone, in order (tested).
 */
typedef struct mtgp_server mtgp_server;

typedef struct mtgp_server_config {
    uint64_t arena_bytes;      /* device memory for outputs, reserved at creation
                                  (0 = 4 GiB)                                       */
    uint64_t chunk;            /* numbers per request per tick (0 = 2^20)         */
    uint32_t max_active;       /* requests generated concurrently (0 = 4096)       */
    uint32_t max_inflight;     /* ticks queued on the GPU at once (0 = 2)          */
} mtgp_server_config;

typedef struct mtgp_completion {
    uint64_t ticket;
    uint32_t gen, dtype;
    uint64_t n;
    void *dev_out;             /* device address of the n outputs (in the arena),
                                  valid until mtgp_server_release(ticket)          */
    double submit_s, done_s;   /* seconds since the server was created: host clock
                                  at submission, device event at completion        */
} mtgp_completion;

typedef struct mtgp_server_stats_t {
    uint32_t pending, active, inflight_ticks;
    uint64_t ticks, numbers_completed, arena_free_bytes;
    double now_s;
} mtgp_server_stats_t;

/* Creates a server over pool p (which it uses exclusively, on `stream`);
 * reserves the arena and captures the tick launch.  Synchronous. */
mtgp_status mtgp_server_create(mtgp_pool *p, const mtgp_server_config *cfg, void *stream, mtgp_server **out);

/* Queues a request; returns its ticket.  MTGP_EINVAL if n == 0, the generator
 * or dtype is out of range, or 4 n bytes exceed the arena.  Host only. */
mtgp_status mtgp_server_submit(mtgp_server *s, uint32_t gen, uint32_t dtype, uint64_t n, uint64_t *ticket);

/* Advances the server (retire, admit, launch one tick if fewer than
 * max_inflight are queued) and returns up to `max` completions in *done.  With
 * block != 0 and nothing else to do, waits for the oldest queued tick. */
mtgp_status mtgp_server_poll(mtgp_server *s, mtgp_completion *done, uint32_t max, uint32_t *ndone, int block);

/* Returns a completed request's arena range to the server. */
mtgp_status mtgp_server_release(mtgp_server *s, uint64_t ticket);

mtgp_status mtgp_server_stats(const mtgp_server *s, mtgp_server_stats_t *out);

/*
 * Native request loop over an arrival trace: submits request i (generator
 * gens[i], dtype dtypes[i], ns[i] numbers) when arrival_s[i] seconds
 * (non-decreasing, from the call) have passed on the host clock, polls, and
 * releases each completed output at once.  Writes each request's latency
 * (device completion minus host submission) to latency_s[i] and, if done_s is
 * not NULL, its completion time since the call.  Returns when all complete.
 * For measuring the served form without a host-language loop in the way.
 */
mtgp_status mtgp_server_run_trace(mtgp_server *s, const double *arrival_s, const uint32_t *gens,
                                  const uint32_t *dtypes, const uint64_t *ns, uint32_t count, double *latency_s,
                                  double *done_s);

/* Waits for queued ticks, then frees the arena, the graph and the server. */
void mtgp_server_destroy(mtgp_server *s);

/* ---- allocation-free form ---------------------------------------------------
 *
 * The paper has no counterpart to this call.  It exists for callers that must
 * not allocate device memory: code running inside a framework whose own
 * allocator already reserves the device's memory, latency-sensitive loops
 * (cudaMalloc and cudaFree can synchronise the whole device), and callers
 * under a fixed memory budget.  Such callers own every buffer and pass it in.
 *
 * Generates, in one launch on `stream`, the requests reqs[0 .. nreq) for the
 * `count` generators with parameter sets ps[0 .. count), blocked layout only
 * (request j writes dev_out[out_offset .. out_offset + n), dtype as in
 * mtgp_request).  Generator i's state is the N_i words at
 * dev_states + state_offsets[i] (x_k .. x_{k+N-1}, oldest first; for example
 * copied from mtgp_pool_read_state); it is read and advanced in place, so
 * the next call continues the streams.  dev_states and dev_out are
 * caller-owned, 4-byte aligned device buffers.
 *
 * Nothing is allocated: the per-call records (parameter tables, work list,
 * error word) go to one file-scope device array of
 * MTGP_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library keeps
 * until the process exits.  count > MTGP_NOALLOC_MAX_GENS or
 * nreq > MTGP_NOALLOC_MAX_REQS returns MTGP_EINVAL with a message.  The first
 * call on each device looks up that array's device address (a one-time
 * set-up; make that first call before any stream capture).  The records are
 * copied out of the call's own host memory, so a stream being captured into a
 * CUDA graph is refused (MTGP_EINVAL).  Every call shares the array and
 * overwrites it (its control words are cleared on each call).  The library
 * holds a lock from a call's copy through its launch, so calls from several
 * host threads on ONE stream queue one after the other and are safe; calls
 * whose work overlaps on the GPU (different streams) race on the array and
 * must not be made.  Overlapping state ranges (two generators sharing words)
 * return MTGP_EINVAL.  The launch shape is sized on the host so that the
 * kernel's buffer check always passes; kernel-side errors therefore cannot
 * occur on this path.  The records are copied from ordinary host memory, so
 * the call may wait for work already queued on `stream` before it returns.
 */
#define MTGP_NOALLOC_SCRATCH_BYTES 32768u
#define MTGP_NOALLOC_MAX_GENS 64u
#define MTGP_NOALLOC_MAX_REQS 64u
mtgp_status mtgp_generate_noalloc(const mtgp_params *ps, uint32_t count, uint32_t *dev_states,
                                  const uint64_t *state_offsets, const mtgp_request *reqs, uint32_t nreq,
                                  void *dev_out, void *stream);

/* ---- measurement helper --------------------------------------------------- */

/*
 * Write-only bandwidth probe: fills `words` 32-bit words of dev_buf with a
 * pattern using 16-byte stores from a grid sized to the SM count; the
 * achievable HBM write rate bounds every generation kernel here (each number
 * costs 4 bytes written and nothing read).  Stream-ordered.
 */
mtgp_status mtgp_fill_probe(void *dev_buf, uint64_t words, uint32_t pattern, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MTGP_H */
