/*
 * MTGP CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the MTGP generation
 * path computes (Saito & Matsumoto, "Variants of Mersenne Twister Suitable for
 * Graphic Processors", arXiv 1005.4973).  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load this code; the product path
 * never does.  It shares no code, header, table or constant generator with the
 * CUDA library: everything here is written out again from the paper.
 *
 * Parity status per function (see the module header of oracle/__init__.py for
 * the pins):
 *   orc_derive / orc_generate          pinned (F2 bit-matrix formulation, linearity,
 *                                      mask invariance, reduced-size period checks,
 *                                      float closed form, continuation)
 *   orc_params_draw / orc_seed_state   project-defined readings of passages the
 *                                      paper leaves open: parity unpinned against any
 *                                      outside source (checked for structure only)
 *   orc_bm / orc_poly_*                pinned against closed forms and brute force
 *   orc_kv                             pinned by the dimension defects the paper
 *                                      prints for MT19937 (Sec. 3.8), the bound
 *                                      k(v) <= floor(p / v) and k(1) = p at full
 *                                      period
 *   orc_mt19937_*                      the published MT19937 (Matsumoto and
 *                                      Nishimura 1998), only as the k(v) pin's input;
 *                                      pinned by ISO C++'s required 10000th output of
 *                                      std::mt19937 and by numpy's MT19937
 *   orc_splitmix64_next / orc_mix64    pinned by the published SplitMix64 outputs for
 *                                      seed 0 (tests/golden/splitmix64_seed0.txt)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_U32 0
#define ORC_F12 1
#define ORC_F01 2

typedef struct {
    uint32_t mexp, N, r, mask, pos, sh1, sh2, id;
    uint32_t R[4];          /* rows of the 4x32 recursion matrix R, row 0 first   */
    uint32_t T[4];          /* rows of the 4x32 tempering matrix T, row 0 first   */
    uint32_t rectbl[16];    /* rectbl[b] = (b as a 4-bit row vector) * R   (Sec. 3.6) */
    uint32_t tmptbl[16];    /* tmptbl[b] = (b as a 4-bit row vector) * T   (Sec. 3.7) */
    uint32_t sngltbl[16];   /* single-precision table of Sec. 6                    */
} orc_params;

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number      */
/* generators", OOPSLA 2014): a Weyl sequence with gamma 0x9E3779B97F4A7C15  */
/* followed by the published 64-bit finaliser.  The paper does not say how   */
/* parameter sets are drawn or states seeded; this published generator is    */
/* the reading taken for both.                                                */
/* ------------------------------------------------------------------------- */
#define ORC_GAMMA 0x9E3779B97F4A7C15ull

uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_next(uint64_t *s)
{
    *s += ORC_GAMMA;
    return orc_mix64(*s);
}

/* BITMASK(w, r) of Sec. 3.6: the w-r MSBs set, the r LSBs clear (w = 32). */
static uint32_t orc_bitmask(uint32_t r)
{
    return r >= 32 ? 0u : (0xFFFFFFFFu << r);
}

/* floor to a power of two, the paper's [x]_2 (Sec. 3.5). */
static uint32_t orc_floor_pow2(uint32_t x)
{
    uint32_t p = 1;
    while (p * 2u <= x) p *= 2u;
    return p;
}

/*
 * Look-up table of a 4x32 matrix (Sec. 3.6, 3.7): entry b is the product of
 * the 4-bit row vector b with the matrix.  The paper writes b in binary with
 * the most significant bit on the left ("0001" is the vector with only its
 * last component set) and identifies a 32-bit word with a row vector whose
 * leftmost component is the MSB (Sec. 5), so the leftmost component of b --
 * bit 3 -- multiplies row 0 and bit 0 multiplies row 3.
 */
void orc_table_from_rows(const uint32_t rows[4], uint32_t tbl[16])
{
    for (uint32_t b = 0; b < 16; b++) {
        uint32_t v = 0;
        for (uint32_t j = 0; j < 4; j++)
            if ((b >> (3u - j)) & 1u) v ^= rows[j];
        tbl[b] = v;
    }
}

/*
 * Fills the derived fields of a parameter set whose mexp, pos, sh1, sh2, id,
 * R and T are set: N = ceil(p / w), r = wN - p (Sec. 3.3), the bit mask
 * (Sec. 3.6), rectbl / tmptbl (Sec. 3.6, 3.7) and sngltbl (Sec. 6).
 *
 * sngltbl: Sec. 6 says each entry has the nine MSBs 001111111 followed by the
 * leading bits of tmptbl[i]; a single-precision word has room for 23 of them,
 * so sngltbl[i] = 0x3F800000 | (tmptbl[i] >> 9).
 */
int orc_derive(orc_params *p)
{
    if (p->mexp < 65u) return -1;
    p->N = (p->mexp + 31u) / 32u;
    p->r = 32u * p->N - p->mexp;
    p->mask = orc_bitmask(p->r);
    if (p->pos < 1u || p->pos >= p->N) return -1;
    if (p->sh1 < 1u || p->sh1 > 31u || p->sh2 < 1u || p->sh2 > 31u) return -1;
    orc_table_from_rows(p->R, p->rectbl);
    orc_table_from_rows(p->T, p->tmptbl);
    for (int b = 0; b < 16; b++) p->sngltbl[b] = 0x3F800000u | (p->tmptbl[b] >> 9);
    return 0;
}

/* Range of the middle position M.  Sec. 5 draws M with 2 < M < N - [N]_2; for
 * states too small for that range to be non-empty, the Sec. 3.5 rule is used:
 * M >= 2 and N - M >= [N - 2]_2. */
void orc_pos_range(uint32_t N, uint32_t *lo, uint32_t *hi)
{
    uint32_t f = orc_floor_pow2(N);
    if (N > f + 3u) { *lo = 3u; *hi = N - f - 1u; return; }
    *lo = 2u;
    *hi = N - orc_floor_pow2(N - 2u);
}

/* The 4x4 matrix acting on the four LSBs of u in the last line of the
 * recursion (Sec. 3.6) is I + R4, R4 being the four LSBs of the rows of R.
 * Sec. 5 (caption of its recursion-parameter figure) requires it invertible. */
int orc_lsb_block_invertible(const uint32_t R[4])
{
    uint32_t m[4];
    for (int j = 0; j < 4; j++)      /* row j of I + R4; component j is bit 3-j */
        m[j] = (R[j] & 0xFu) ^ (1u << (3 - j));
    int rank = 0;
    for (int bit = 3; bit >= 0; bit--) {
        int piv = -1;
        for (int j = rank; j < 4; j++)
            if ((m[j] >> bit) & 1u) { piv = j; break; }
        if (piv < 0) continue;
        uint32_t t = m[piv]; m[piv] = m[rank]; m[rank] = t;
        for (int j = 0; j < 4; j++)
            if (j != rank && ((m[j] >> bit) & 1u)) m[j] ^= m[rank];
        rank++;
    }
    return rank == 4;
}

/*
 * Draws a synthetic parameter set with the structure MTGPDC gives its sets
 * (Sec. 5): ID[31:16] in the 16 MSBs of row 0 of R; ID[15:0] in row 1, in the
 * sixteen bit positions 13..28 counted from the MSB (bits 19..4); the four
 * LSBs of every row redrawn until I + R4 is invertible; every other bit of R
 * random; sh1 = 13, sh2 = 4; M uniform in the range above.  T is random.
 *
 * Draw order (SplitMix64 stream started at param_seed): M; R rows 0..3; the
 * LSB nibbles of rows 0..3 again for every rejected attempt; T rows 0..3;
 * then, only if random_shifts != 0, sh1 and sh2 uniform in [1, 31].
 * The paper does not fix this procedure: parity unpinned against MTGPDC.
 */
int orc_params_draw(uint32_t mexp, uint64_t param_seed, uint32_t id,
                    int random_shifts, orc_params *out)
{
    memset(out, 0, sizeof *out);
    if (mexp < 65u) return -1;
    uint64_t s = param_seed;
    uint32_t N = (mexp + 31u) / 32u, lo, hi;
    orc_pos_range(N, &lo, &hi);
    if (hi < lo) return -1;
    out->mexp = mexp;
    out->id = id;
    out->pos = lo + (uint32_t)(orc_splitmix64_next(&s) % (uint64_t)(hi - lo + 1u));
    for (int j = 0; j < 4; j++) out->R[j] = (uint32_t)orc_splitmix64_next(&s);
    out->R[0] = (out->R[0] & 0x0000FFFFu) | (id & 0xFFFF0000u);
    out->R[1] = (out->R[1] & ~0x000FFFF0u) | ((id & 0x0000FFFFu) << 4);
    while (!orc_lsb_block_invertible(out->R))
        for (int j = 0; j < 4; j++)
            out->R[j] = (out->R[j] & ~0xFu) | ((uint32_t)orc_splitmix64_next(&s) & 0xFu);
    for (int j = 0; j < 4; j++) out->T[j] = (uint32_t)orc_splitmix64_next(&s);
    out->sh1 = 13u;
    out->sh2 = 4u;
    if (random_shifts) {
        out->sh1 = 1u + (uint32_t)(orc_splitmix64_next(&s) % 31u);
        out->sh2 = 1u + (uint32_t)(orc_splitmix64_next(&s) % 31u);
    }
    return orc_derive(out);
}

/*
 * Initial state x_0 .. x_{N-1} of generator gen_id from a 64-bit seed.  The
 * paper only says the host initialises the state array (Sec. 8); the reading
 * taken: key = first SplitMix64 output of the stream started at gen_id; word j
 * is the low 32 bits of output j+1 of the stream started at seed ^ key.  The
 * state is all zero in its p effective bits with probability 2^-p; that state
 * is a fixed point, so then x_{N-1} is set to 1.  Parity unpinned (project
 * definition).
 */
void orc_seed_state(const orc_params *p, uint32_t gen_id, uint64_t seed, uint32_t *state)
{
    uint64_t g = gen_id;
    uint64_t key = orc_splitmix64_next(&g);
    uint64_t s = seed ^ key;
    uint32_t any = 0;
    for (uint32_t j = 0; j < p->N; j++) {
        state[j] = (uint32_t)orc_splitmix64_next(&s);
        any |= (j == 0) ? (state[j] & p->mask) : state[j];
    }
    if (!any) state[p->N - 1] = 1u;
}

static uint32_t orc_f32_bits_minus_one(uint32_t bits)
{
    union { uint32_t u; float f; } a;
    a.u = bits;
    volatile float f = a.f;   /* one IEEE single subtraction, no contraction */
    a.f = f - 1.0f;
    return a.u;
}

/*
 * Generates n outputs of one generator and advances its state, following the
 * paper's definitions literally on a straight array x[0 .. N+n) (no ring):
 *   recursion (Definition of Sec. 3.6, C form):
 *     t = x[k+1] ^ (x[k] & BITMASK);  t ^= t << sh1;
 *     u = t ^ (x[k+M] >> sh2);         x[N+k] = u ^ rectbl[u & 0xf];
 *   tempering (Definition of Sec. 3.7, C form), output o_{N+k}:
 *     t = x[M-1+k] ^ (x[M-1+k] >> 16); t ^= t >> 8;
 *     o = x[N+k] ^ tmptbl[t & 0xf];
 *   single precision (Sec. 6, eq. C): the last line becomes
 *     o = (x[N+k] >> 9) ^ sngltbl[t & 0xf]      -- a float in [1, 2)
 *   and [0, 1) is that float minus 1.0 in single precision.
 * The k-th output of a call is o_{N+k}: the N state words are never output.
 * On return state[] holds x[n .. n+N), so the next call continues the stream
 * (Sec. 8: the state is written back after every call).
 * Outputs are written as 32-bit patterns (uint32 or the float's bits).
 */
int orc_generate(const orc_params *p, uint32_t *state, uint64_t n, int dtype, uint32_t *out)
{
    const uint64_t N = p->N, M = p->pos;
    uint32_t *x = (uint32_t *)malloc((size_t)(N + n) * sizeof(uint32_t));
    if (!x) return -1;
    memcpy(x, state, (size_t)N * sizeof(uint32_t));
    for (uint64_t k = 0; k < n; k++) {
        uint32_t t = x[k + 1] ^ (x[k] & p->mask);
        t ^= t << p->sh1;
        uint32_t u = t ^ (x[k + M] >> p->sh2);
        x[N + k] = u ^ p->rectbl[u & 0xfu];
    }
    for (uint64_t k = 0; k < n; k++) {
        uint32_t t = x[M - 1 + k] ^ (x[M - 1 + k] >> 16);
        t ^= t >> 8;
        if (dtype == ORC_U32) {
            out[k] = x[N + k] ^ p->tmptbl[t & 0xfu];
        } else {
            uint32_t bits = (x[N + k] >> 9) ^ p->sngltbl[t & 0xfu];
            out[k] = (dtype == ORC_F01) ? orc_f32_bits_minus_one(bits) : bits;
        }
    }
    memcpy(state, x + n, (size_t)N * sizeof(uint32_t));
    free(x);
    return 0;
}

/* ---- many generators on the host cores: one generator per thread -------- */
typedef struct {
    const orc_params *params;
    uint32_t **states;
    uint32_t **outs;
    const uint64_t *ns;
    const int *dtypes;
    int count, next, err;
    pthread_mutex_t mu;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *j = (orc_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->count) break;
        if (orc_generate(&j->params[i], j->states[i], j->ns[i], j->dtypes[i], j->outs[i]))
            j->err = 1;
    }
    return NULL;
}

/* Runs orc_generate for count independent generators on nthreads threads. */
int orc_generate_many(const orc_params *params, uint32_t **states, const uint64_t *ns,
                      const int *dtypes, uint32_t **outs, int count, int nthreads)
{
    orc_job j = { params, states, outs, ns, dtypes, count, 0, 0 };
    pthread_mutex_init(&j.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, orc_worker, &j);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&j.mu);
    return j.err ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* F2 tools for the reduced-size structural checks (Sec. 3.3, Sec. 5).       */
/* Polynomials over F2 are bit arrays: bit i of word i/64 = coefficient x^i. */
/* ------------------------------------------------------------------------- */

/*
 * Berlekamp-Massey over F2 (the minimal-polynomial step of Sec. 5).  Input:
 * bits s[0 .. n).  Output: L and the minimal polynomial
 *   phi(x) = x^L + c_1 x^(L-1) + ... + c_L,  s_k = sum_i c_i s_{k-i},
 * written to poly[0 .. L] as bytes (poly[i] = coefficient of x^i).
 */
int orc_bm(const uint8_t *s, int n, uint8_t *poly)
{
    uint8_t *C = (uint8_t *)calloc((size_t)n + 1, 1);
    uint8_t *B = (uint8_t *)calloc((size_t)n + 1, 1);
    uint8_t *T = (uint8_t *)calloc((size_t)n + 1, 1);
    int L = 0, m = 1;
    C[0] = B[0] = 1;
    for (int k = 0; k < n; k++) {
        uint8_t d = s[k];
        for (int i = 1; i <= L; i++) d ^= (uint8_t)(C[i] & s[k - i]);
        if (!d) { m++; continue; }
        if (2 * L <= k) {
            memcpy(T, C, (size_t)n + 1);
            for (int i = 0; i + m <= n; i++) C[i + m] ^= B[i];
            L = k + 1 - L;
            memcpy(B, T, (size_t)n + 1);
            m = 1;
        } else {
            for (int i = 0; i + m <= n; i++) C[i + m] ^= B[i];
            m++;
        }
    }
    /* connection polynomial C(x) = 1 + c_1 x + ... ; minimal poly = x^L C(1/x) */
    for (int i = 0; i <= L; i++) poly[i] = C[L - i];
    free(C); free(B); free(T);
    return L;
}

static int orc_words(int bits) { return (bits + 63) / 64; }

/* a <- a mod f, a of degree < abits, f monic of degree deg (bit arrays). */
static void orc_poly_reduce(uint64_t *a, int abits, const uint64_t *f, int deg)
{
    int fw = orc_words(deg + 1), aw = orc_words(abits);
    for (int i = abits - 1; i >= deg; i--) {
        if (!((a[i >> 6] >> (i & 63)) & 1u)) continue;
        int sh = i - deg, ws = sh >> 6, bs = sh & 63;   /* a ^= f << sh */
        for (int q = 0; q < fw; q++) {
            uint64_t v = f[q];
            if (q + ws < aw) a[q + ws] ^= v << bs;
            if (bs && q + ws + 1 < aw) a[q + ws + 1] ^= v >> (64 - bs);
        }
    }
}

/*
 * Irreducibility test for a degree-p polynomial f over F2 with p prime (a
 * Mersenne exponent): f is irreducible iff x^(2^p) = x mod f and f has no
 * root in F2 (the only factor degrees that divide p are 1 and p).  With p a
 * Mersenne exponent, irreducible implies primitive (Sec. 5).
 * poly[0 .. deg] are bytes.  Returns 1 if irreducible.
 */
int orc_poly_irreducible_prime(const uint8_t *poly, int deg)
{
    if (deg < 2 || !poly[deg]) return 0;
    if (!poly[0]) return 0;                      /* root 0 */
    int ones = 0;
    for (int i = 0; i <= deg; i++) ones ^= poly[i];
    if (!ones) return 0;                         /* root 1 */
    int w = orc_words(deg + 1), w2 = orc_words(2 * deg + 1);
    uint64_t *f = (uint64_t *)calloc((size_t)w, 8);
    uint64_t *a = (uint64_t *)calloc((size_t)w2, 8);
    uint64_t *sq = (uint64_t *)calloc((size_t)w2, 8);
    for (int i = 0; i <= deg; i++) if (poly[i]) f[i >> 6] |= 1ull << (i & 63);
    a[0] = 2u;                                   /* the polynomial x */
    for (int it = 0; it < deg; it++) {           /* a <- a^2 mod f */
        memset(sq, 0, (size_t)w2 * 8);
        for (int i = 0; i < deg; i++)
            if ((a[i >> 6] >> (i & 63)) & 1u) sq[(2 * i) >> 6] |= 1ull << ((2 * i) & 63);
        orc_poly_reduce(sq, 2 * deg - 1, f, deg);
        memcpy(a, sq, (size_t)w * 8);
        memset(a + w, 0, (size_t)(w2 - w) * 8);
    }
    uint64_t *xx = (uint64_t *)calloc((size_t)w2, 8);
    xx[0] = 2u;
    int ok = memcmp(a, xx, (size_t)w * 8) == 0;
    free(f); free(a); free(sq); free(xx);
    return ok;
}

/* ---- dense F2 matrices, rows packed into 64-bit words -------------------- */

/* C = A * B for n x n matrices with rows of w = ceil(n/64) words. */
void orc_f2mat_mul(const uint64_t *A, const uint64_t *B, uint64_t *C, int n)
{
    int w = orc_words(n);
    memset(C, 0, (size_t)n * (size_t)w * 8);
    for (int i = 0; i < n; i++) {
        const uint64_t *a = A + (size_t)i * w;
        uint64_t *c = C + (size_t)i * w;
        for (int k = 0; k < n; k++)
            if ((a[k >> 6] >> (k & 63)) & 1u) {
                const uint64_t *b = B + (size_t)k * w;
                for (int q = 0; q < w; q++) c[q] ^= b[q];
            }
    }
}

/* Rank over F2 of an n x n packed matrix (copied). */
int orc_f2mat_rank(const uint64_t *A, int n)
{
    int w = orc_words(n), rank = 0;
    uint64_t *m = (uint64_t *)malloc((size_t)n * (size_t)w * 8);
    memcpy(m, A, (size_t)n * (size_t)w * 8);
    for (int col = 0; col < n && rank < n; col++) {
        int piv = -1;
        for (int i = rank; i < n; i++)
            if ((m[(size_t)i * w + (col >> 6)] >> (col & 63)) & 1u) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int q = 0; q < w; q++) {
                uint64_t t = m[(size_t)piv * w + q];
                m[(size_t)piv * w + q] = m[(size_t)rank * w + q];
                m[(size_t)rank * w + q] = t;
            }
        for (int i = 0; i < n; i++)
            if (i != rank && ((m[(size_t)i * w + (col >> 6)] >> (col & 63)) & 1u))
                for (int q = 0; q < w; q++) m[(size_t)i * w + q] ^= m[(size_t)rank * w + q];
        rank++;
    }
    free(m);
    return rank;
}

/* out = F^(2^k) by k squarings. */
void orc_f2mat_pow2k(const uint64_t *F, uint64_t *out, int n, int k)
{
    int w = orc_words(n);
    size_t bytes = (size_t)n * (size_t)w * 8;
    uint64_t *tmp = (uint64_t *)malloc(bytes);
    memcpy(out, F, bytes);
    for (int i = 0; i < k; i++) {
        orc_f2mat_mul(out, out, tmp, n);
        memcpy(out, tmp, bytes);
    }
    free(tmp);
}

/* out = phi(F) by Horner's rule; poly[0..deg] bytes, coefficient of x^i. */
void orc_f2mat_polyeval(const uint8_t *poly, int deg, const uint64_t *F, uint64_t *out, int n)
{
    int w = orc_words(n);
    size_t bytes = (size_t)n * (size_t)w * 8;
    uint64_t *tmp = (uint64_t *)malloc(bytes);
    memset(out, 0, bytes);
    for (int d = deg; d >= 0; d--) {
        orc_f2mat_mul(out, F, tmp, n);
        memcpy(out, tmp, bytes);
        if (poly[d])
            for (int i = 0; i < n; i++) out[(size_t)i * w + (i >> 6)] ^= 1ull << (i & 63);
    }
    free(tmp);
}

/*
 * Small-size MTGPDC recursion search (Sec. 5): draw parameter sets with the
 * given ID (param seeds seed0, seed0+1, ...) until the minimal polynomial of
 * the MSB sequence of x_k -- found by Berlekamp-Massey over 2p bits -- has
 * degree p and is irreducible.  Returns the number of candidates tried, or -1
 * if none of max_tries qualified.  Sizes with p of a few thousand at most.
 */
int orc_search_full_period(uint32_t mexp, uint64_t seed0, uint32_t id, int max_tries,
                           orc_params *out, uint64_t *found_seed)
{
    int nb = 2 * (int)mexp;
    uint8_t *bits = (uint8_t *)malloc((size_t)nb);
    uint8_t *poly = (uint8_t *)malloc((size_t)nb + 1);
    int ret = -1;
    for (int t = 0; t < max_tries; t++) {
        orc_params p;
        if (orc_params_draw(mexp, seed0 + (uint64_t)t, id, 0, &p)) break;
        uint32_t *st = (uint32_t *)malloc(p.N * 4u);
        uint32_t *x = (uint32_t *)malloc(((size_t)p.N + (size_t)nb) * 4u);
        orc_seed_state(&p, 0, 12345u + (uint64_t)t, st);
        memcpy(x, st, p.N * 4u);
        const uint64_t N = p.N, M = p.pos;
        for (uint64_t k = 0; k < (uint64_t)nb; k++) {
            uint32_t tt = x[k + 1] ^ (x[k] & p.mask);
            tt ^= tt << p.sh1;
            uint32_t u = tt ^ (x[k + M] >> p.sh2);
            x[N + k] = u ^ p.rectbl[u & 0xfu];
            bits[k] = (uint8_t)(x[N + k] >> 31);
        }
        free(st); free(x);
        int L = orc_bm(bits, nb, poly);
        if (L == (int)mexp && orc_poly_irreducible_prime(poly, L)) {
            *out = p;
            *found_seed = seed0 + (uint64_t)t;
            ret = t + 1;
            break;
        }
    }
    free(bits); free(poly);
    return ret;
}

/* ---- dimensions of equidistribution (Sec. 3.4, 3.8) ---------------------- */

/*
 * k(v) for v = 1 .. vmax of a 32-bit output sequence seq[0 .. L) of an
 * F2-linear generator with state dimension p, period 2^p - 1 and seq taken
 * from a nonzero state s.  The v-bit MSB sequence is k-dimensionally
 * equidistributed iff the linear map from states to the v MSBs of k
 * consecutive outputs is onto, i.e. has rank k v.  The states F^j s
 * (j = 0 .. p-1) form a basis (s is cyclic at full period), so the map's
 * matrix in that basis has the row (i, b) = bit b of seq[i + j], j < p.
 * Rows are added output by output (v rows each, MSB first) to a row-echelon
 * basis kept by lowest set bit; k(v) is the number of outputs before the
 * first dependent row.  Needs L >= p + floor(p / v) + 1.  Returns 0, or -1
 * on allocation failure.
 */
int orc_kv(const uint32_t *seq, int L, int p, int vmax, int *kv)
{
    const int W = (p + 63) / 64;
    uint64_t *basis = (uint64_t *)malloc((size_t)p * (size_t)W * 8u);
    int *piv = (int *)malloc((size_t)p * sizeof(int));
    uint64_t *row = (uint64_t *)malloc((size_t)W * 8u);
    if (!basis || !piv || !row) { free(basis); free(piv); free(row); return -1; }
    for (int v = 1; v <= vmax; v++) {
        for (int c = 0; c < p; c++) piv[c] = -1;
        int rank = 0, k = 0, dependent = 0;
        for (int i = 0; !dependent && i + p <= L; i++) {
            for (int b = 31; b > 31 - v && !dependent; b--) {
                memset(row, 0, (size_t)W * 8u);
                for (int j = 0; j < p; j++)
                    if ((seq[i + j] >> b) & 1u) row[j >> 6] |= 1ull << (j & 63);
                for (;;) {
                    int c = -1;
                    for (int w = 0; w < W; w++)
                        if (row[w]) { c = 64 * w + __builtin_ctzll(row[w]); break; }
                    if (c < 0) { dependent = 1; break; }
                    if (piv[c] < 0) {
                        memcpy(basis + (size_t)rank * W, row, (size_t)W * 8u);
                        piv[c] = rank++;
                        break;
                    }
                    const uint64_t *r = basis + (size_t)piv[c] * W;
                    for (int w = 0; w < W; w++) row[w] ^= r[w];
                }
            }
            if (!dependent) k = i + 1;
        }
        kv[v - 1] = k;
    }
    free(basis); free(piv); free(row);
    return 0;
}

/*
 * The published MT19937 (Matsumoto and Nishimura, ACM TOMACS 1998): N = 624,
 * M = 397, r = 31 (one upper bit of x_i joins the 31 lower bits of x_{i+1}),
 * twist vector 0x9908b0df; tempering shifts 11, 7, 15, 18 with masks
 * 0x9d2c5680 and 0xefc60000.  State filled by SplitMix64 from `seed` (any
 * nonzero state will do for orc_kv).  Straight array, n outputs.
 */
/* The published MT19937 seeding by one 32-bit integer (Matsumoto and
 * Nishimura's init_genrand): x_0 = s, x_j = 1812433253 (x_{j-1} xor
 * (x_{j-1} >> 30)) + j mod 2^32.  With s = 5489 it is the state of a
 * default-constructed std::mt19937 in ISO C++. */
void orc_mt19937_init_genrand(uint32_t s, uint32_t *x624)
{
    x624[0] = s;
    for (uint32_t j = 1; j < 624u; j++)
        x624[j] = 1812433253u * (x624[j - 1] ^ (x624[j - 1] >> 30)) + j;
}

/* n outputs of MT19937 from the 624-word state x624 (oldest word first). */
int orc_mt19937_outputs_from(const uint32_t *x624, int n, uint32_t *out)
{
    const int N = 624, M = 397;
    uint32_t *x = (uint32_t *)malloc(((size_t)N + (size_t)n) * 4u);
    if (!x) return -1;
    memcpy(x, x624, (size_t)N * 4u);
    for (int i = 0; i < n; i++) {
        const uint32_t y = (x[i] & 0x80000000u) | (x[i + 1] & 0x7fffffffu);
        x[N + i] = x[i + M] ^ (y >> 1) ^ ((y & 1u) ? 0x9908b0dfu : 0u);
        uint32_t z = x[N + i];
        z ^= z >> 11;
        z ^= (z << 7) & 0x9d2c5680u;
        z ^= (z << 15) & 0xefc60000u;
        z ^= z >> 18;
        out[i] = z;
    }
    free(x);
    return 0;
}

/* n outputs of MT19937 from a state of SplitMix64 words keyed by `seed` (any
 * nonzero state serves the k(v) pin, which does not depend on the state). */
int orc_mt19937_outputs(uint64_t seed, int n, uint32_t *out)
{
    uint32_t x[624];
    uint64_t s = seed;
    for (int j = 0; j < 624; j++) x[j] = (uint32_t)orc_splitmix64_next(&s);
    x[0] |= 0x80000000u;                          /* the upper bit of x_0 is state: nonzero */
    return orc_mt19937_outputs_from(x, n, out);
}

/* Size of the parameter struct, so the Python side can check its mirror. */
int orc_params_sizeof(void) { return (int)sizeof(orc_params); }
