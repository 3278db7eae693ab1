/*
 * asse_oracle.c -- plain, slow CPU oracle of the ASSE sliding-window
 * super-point method (Xu, "Distributed super point cardinality estimation
 * under sliding time window for high speed network", arXiv 1807.01527).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  The product
 * path (the CUDA library under paper_1807_01527_gb300/) never calls it, and
 * the two share no code: different hash code, different state layout (here
 * one byte per AT, there packed 32-bit words), different restore algorithm.
 *
 * Every function below follows one passage of the paper, named in its
 * comment.  Where the paper is silent or garbled, the reading taken is stated
 * beside the code.  All arithmetic on AT values and hashes is exact integer;
 * the estimates of Eq.2/Eq.4 are evaluated in double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The mangling modulus p of f(aip) = A*aip mod p (Sec. 2.5 and Sec. 4.1): a
 * prime just above 2^32.  Reading: p = 2^32 + 15, the smallest such prime. */
#define ORACLE_P 4294967311ULL
#define TWO32 4294967296ULL

typedef struct {
    uint32_t k;      /* window size in slices: AT values 0..2k, 2k = inactive */
    uint32_t theta;  /* super point threshold */
    uint32_t g;      /* ATs per ATV (bits per linear estimator) */
    uint32_t r;      /* rows of the ATV cube */
    uint32_t c;      /* column-index bits per row */
    uint32_t u;      /* frame bits */
    uint32_t s;      /* start offset between consecutive rows' column windows */
    uint32_t A;      /* mangling multiplier, 2 <= A < 2^32 */
    uint64_t bh_a;   /* BH multiplier (odd) */
    uint64_t bh_b;   /* BH offset */
    uint32_t mode;   /* 0: asynchronous timestamps (Sec. 3); 1: aging counter ACE (Sec. 2.3);
                      * 2: asynchronous timestamps with one ACT shared by the whole ATV */
    uint32_t pad;
} oracle_params;

typedef struct {
    oracle_params p;
    uint32_t E;     /* ATVs per row: 2^(c+u) */
    uint32_t W;     /* width of LBS(f(aip), 32-u) */
    uint64_t Ainv;  /* A^-1 mod p */
    uint64_t t;     /* index of the open slice (0-based) */
    uint8_t *at;    /* counter values, [r][E][g], one byte each */
} oracle_state;

/* ---------------------------------------------------------------- Sec. 3 */

/* Algorithm 1 (checkAT): an AT with value 2k is inactive; otherwise it is
 * active for the latest k' slices iff its distance to its ACT,
 * (act + 2k - value) mod 2k, is at most k'-1. */
int oracle_check_at(uint32_t value, uint32_t act, uint32_t k, uint32_t kp)
{
    if (value == 2 * k)
        return 0;
    uint32_t dis = (act + 2 * k - value) % (2 * k);
    return dis <= kp - 1;
}

/* Algorithm 2 (preserveAT), applied at the beginning of a slice with the
 * AT's new ACT.  Only ACT values 0 and k do anything.  At ACT 0 the values
 * 0..k become 2k; at ACT k the values k..2k-1 and the value 0 become 2k.
 * The clear of value 0 at ACT 0 is kept although ACT k already cleared it. */
uint32_t oracle_preserve_at(uint32_t value, uint32_t act, uint32_t k)
{
    if (act % k != 0)
        return value;
    if (act == 0) {
        if (value <= k)
            value = 2 * k;
    }
    if (act == k) {
        if (value >= k && value <= 2 * k - 1)
            value = 2 * k;
        if (value == 0)
            value = 2 * k;
    }
    return value;
}

/* Sec. 3, ATV: the g ATs form 2k blocks, the first 2k-1 of a ATs each and the
 * last of b = g - a(2k-1).  Reading: a = floor(g / 2k), blocks contiguous in
 * AT index, so AT h is in block min(h / a, 2k-1). */
uint32_t oracle_block(const oracle_state *st, uint32_t h)
{
    /* Aligned variant (mode 2): the ATV is one block, so every AT has ACT C0
     * and the whole pool is checked by preserveAT once every k slices
     * instead of two of 2k blocks every slice. */
    if (st->p.mode == 2)
        return 0;
    uint32_t a = st->p.g / (2 * st->p.k);
    uint32_t b = h / a;
    return b < 2 * st->p.k - 1 ? b : 2 * st->p.k - 1;
}

/* Sec. 3, ATV: block i has ACT (C0 + i) mod 2k, where C0, the ACT of the
 * first block, advances by one per slice.  Reading: C0 = t mod 2k for the
 * 0-based slice t. */
uint32_t oracle_act(const oracle_state *st, uint32_t h)
{
    uint32_t k2 = 2 * st->p.k;
    uint32_t c0 = (uint32_t)(st->t % k2);
    return (c0 + oracle_block(st, h)) % k2;
}

/* ---------------------------------------------------------------- Sec. 4.1 */

static uint64_t mulmod_p(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * b) % ORACLE_P);
}

/* f(aip) = A*aip mod p (Sec. 4.1).  A value of A*aip mod p at or above 2^32
 * does not fit the 32 bits that RRH slices, so f multiplies again until it
 * lands below 2^32 (cycle walking), which keeps f one-to-one on 32-bit
 * addresses. */
uint32_t oracle_mangle(const oracle_state *st, uint32_t aip)
{
    uint64_t y = mulmod_p(st->p.A, aip);
    while (y >= TWO32)
        y = mulmod_p(st->p.A, y);
    return (uint32_t)y;
}

/* f^-1(y) = A^-1 * y mod p (Sec. 4.1), with the same cycle walk. */
uint32_t oracle_unmangle(const oracle_state *st, uint32_t y)
{
    uint64_t x = mulmod_p(st->Ainv, y);
    while (x >= TWO32)
        x = mulmod_p(st->Ainv, x);
    return (uint32_t)x;
}

/* A^-1 mod p by the extended Euclidean algorithm. */
static uint64_t inverse_mod_p(uint64_t a)
{
    int64_t t0 = 0, t1 = 1;
    int64_t r0 = (int64_t)ORACLE_P, r1 = (int64_t)a;
    while (r1 != 0) {
        int64_t q = r0 / r1, tmp;
        tmp = r0 - q * r1; r0 = r1; r1 = tmp;
        tmp = t0 - q * t1; t0 = t1; t1 = tmp;
    }
    if (t0 < 0)
        t0 += (int64_t)ORACLE_P;
    return (uint64_t)t0;
}

uint64_t oracle_inverse_A(const oracle_state *st) { return st->Ainv; }

/* Bit n of LBS(f, W), counted from the left (n = 0 is the most significant
 * of the W bits). */
static uint32_t lbs_bit(uint32_t L, uint32_t W, uint32_t n)
{
    return (L >> (W - 1 - n)) & 1u;
}

/* RRH(aip) (Sec. 4.1): Z = RBS(f, u) is the frame; x_i takes c successive
 * bits of LBS(f, 32-u) starting at position s*i, wrapping past the last
 * position to position 0.  x_i[0] (the first bit taken) is the most
 * significant bit of x_i. */
void oracle_rrh(const oracle_state *st, uint32_t aip, uint32_t *x, uint32_t *z)
{
    uint32_t f = oracle_mangle(st, aip);
    uint32_t u = st->p.u, W = st->W;
    *z = (uint32_t)((uint64_t)f & ((1ULL << u) - 1));
    uint32_t L = (uint32_t)((uint64_t)f >> u);
    for (uint32_t i = 0; i < st->p.r; i++) {
        uint32_t xi = 0;
        for (uint32_t n = 0; n < st->p.c; n++) {
            uint32_t pos = (st->p.s * i + n) % W;
            xi = (xi << 1) | lbs_bit(L, W, pos);
        }
        x[i] = xi;
    }
}

/* BH(bip) (Sec. 3 and Sec. 4.1) maps bip to [0, g-1]; the paper leaves the
 * family open.  Reading: multiply-add-shift, the top 32 bits of
 * (bh_a*bip + bh_b) mod 2^64, scaled to [0, g) by a 32x32 high product. */
uint32_t oracle_bh(const oracle_state *st, uint32_t bip)
{
    uint64_t h = st->p.bh_a * (uint64_t)bip + st->p.bh_b;
    uint32_t hi = (uint32_t)(h >> 32);
    return (uint32_t)(((uint64_t)hi * st->p.g) >> 32);
}

/* ------------------------------------------------------------ state */

static size_t at_index(const oracle_state *st, uint32_t row, uint32_t est, uint32_t h)
{
    return ((size_t)row * st->E + est) * st->p.g + h;
}

static uint32_t inactive_value(const oracle_state *st)
{
    return st->p.mode == 1 ? 0 : 2 * st->p.k;
}

/* InitAT on every AT of the ATV cube (Sec. 3, Sec. 4). */
oracle_state *oracle_create(const oracle_params *p)
{
    if (p->k < 1 || p->k > 127 || p->g < 2 * p->k || p->r < 1 || p->r > 32 || p->c < 1 || p->u > 8 ||
        p->c + p->u > 24 || p->c > 32 - p->u || p->A < 2 || p->mode > 2)
        return NULL;
    oracle_state *st = (oracle_state *)calloc(1, sizeof(*st));
    if (!st)
        return NULL;
    st->p = *p;
    st->E = 1u << (p->c + p->u);
    st->W = 32 - p->u;
    st->Ainv = inverse_mod_p(p->A);
    st->t = 0;
    size_t n = (size_t)p->r * st->E * p->g;
    st->at = (uint8_t *)malloc(n);
    if (!st->at) {
        free(st);
        return NULL;
    }
    memset(st->at, (int)inactive_value(st), n);
    return st;
}

void oracle_destroy(oracle_state *st)
{
    if (st) {
        free(st->at);
        free(st);
    }
}

uint8_t *oracle_at(oracle_state *st) { return st->at; }
uint64_t oracle_slice(const oracle_state *st) { return st->t; }
uint32_t oracle_num_atv(const oracle_state *st) { return st->E; }

/* Algorithm 3 (Scan IP pair): for each of the r tuples of RRH(aip), SetAT
 * on AT BH(bip) of that ATV, i.e. store the AT's ACT.  In the aging-counter
 * mode (ACE, Sec. 2.3) a visit stores the maximum value k instead. */
void oracle_ingest(oracle_state *st, const uint32_t *pairs, uint64_t n)
{
    uint32_t x[32], z;
    for (uint64_t q = 0; q < n; q++) {
        uint32_t aip = pairs[2 * q], bip = pairs[2 * q + 1];
        oracle_rrh(st, aip, x, &z);
        uint32_t h = oracle_bh(st, bip);
        for (uint32_t i = 0; i < st->p.r; i++) {
            uint32_t est = (z << st->p.c) | x[i];
            uint32_t v = st->p.mode == 1 ? st->p.k : oracle_act(st, h);
            st->at[at_index(st, i, est, h)] = (uint8_t)v;
        }
    }
}

/* Close the open slice and open the next one.  AT mode: the ACT of every
 * block advances and preserveAT (Algorithm 2) runs on every AT at the
 * beginning of the new slice (applying it to ATs whose ACT is neither 0 nor
 * k is a no-op).  ACE mode: at the end of a slice every non-zero aging
 * counter is decremented by one (Sec. 2.3). */
void oracle_advance(oracle_state *st)
{
    uint32_t k = st->p.k;
    if (st->p.mode == 1) {
        size_t n = (size_t)st->p.r * st->E * st->p.g;
        for (size_t q = 0; q < n; q++)
            if (st->at[q] != 0)
                st->at[q] -= 1;
        st->t += 1;
        return;
    }
    st->t += 1;
    for (uint32_t i = 0; i < st->p.r; i++)
        for (uint32_t e = 0; e < st->E; e++)
            for (uint32_t h = 0; h < st->p.g; h++) {
                size_t q = at_index(st, i, e, h);
                st->at[q] = (uint8_t)oracle_preserve_at(st->at[q], oracle_act(st, h), k);
            }
}

/* Active test of one counter for the latest k' slices: Algorithm 1 in AT
 * mode.  ACE mode: a counter visited d slices ago holds k-d, so it is active
 * for k' slices iff its value is at least k-k'+1 (the paper's "no less than
 * c-k-1" read as this k'-slice condition). */
int oracle_active(const oracle_state *st, uint32_t row, uint32_t est, uint32_t h, uint32_t kp)
{
    uint32_t v = st->at[at_index(st, row, est, h)];
    if (st->p.mode == 1)
        return v >= st->p.k - kp + 1;
    return oracle_check_at(v, oracle_act(st, h), st->p.k, kp);
}

/* |ATV|^{k'} (Sec. 3): the number of active ATs of every ATV, [r][E]. */
void oracle_counts(const oracle_state *st, uint32_t kp, uint32_t *cnt)
{
    for (uint32_t i = 0; i < st->p.r; i++)
        for (uint32_t e = 0; e < st->E; e++) {
            uint32_t n = 0;
            for (uint32_t h = 0; h < st->p.g; h++)
                n += (uint32_t)oracle_active(st, i, e, h, kp);
            cnt[(size_t)i * st->E + e] = n;
        }
}

/* |AAT(k', i, j)| (Sec. 4.3): active ATs of row i, frame j, [r][2^u]. */
void oracle_aat(const oracle_state *st, const uint32_t *cnt, uint64_t *aat)
{
    uint32_t nf = 1u << st->p.u, cols = 1u << st->p.c;
    for (uint32_t i = 0; i < st->p.r; i++)
        for (uint32_t j = 0; j < nf; j++) {
            uint64_t s = 0;
            for (uint32_t x = 0; x < cols; x++)
                s += cnt[(size_t)i * st->E + (((size_t)j << st->p.c) | x)];
            aat[(size_t)i * nf + j] = s;
        }
}

/* Super ATV threshold (Sec. 4.2): an ATV is super when |ATV|^{k'} is no
 * smaller than g - g*exp(-theta/g).  Counts are integers, so the test is
 * count >= ceil(g - g*exp(-theta/g)). */
uint32_t oracle_threshold(const oracle_state *st)
{
    double g = (double)st->p.g;
    return (uint32_t)ceil(g - g * exp(-(double)st->p.theta / g));
}

/* Column windows of RRH as bit masks over LBS: the W-bit value whose
 * positions covered by x_i carry x_i's bits, and the mask of those
 * positions. */
static void place(const oracle_state *st, uint32_t i, uint32_t xi, uint32_t *val, uint32_t *mask)
{
    uint32_t W = st->W, c = st->p.c, v = 0, m = 0;
    for (uint32_t n = 0; n < c; n++) {
        uint32_t pos = (st->p.s * i + n) % W;
        uint32_t bit = (xi >> (c - 1 - n)) & 1u;
        v |= bit << (W - 1 - pos);
        m |= 1u << (W - 1 - pos);
    }
    *val = v;
    *mask = m;
}

/* Algorithm 4 (Restore candidate super point).  For every frame j (reading:
 * j runs over all 2^u frames, and CSIP is returned once after the last
 * frame), every column tuple of SA(0,j) x ... x SA(r-1,j) is checked on its
 * duplicate positions: the bits that x_i and x_{(i+1) mod r} place on a
 * position both cover must agree, for every i; a tuple failing any check is
 * dropped (reading of the garbled "Continue").  A passing tuple gives LBS
 * (each position's bit from a row covering it), RBS = j, and the candidate
 * f^-1(LBS . RBS).
 *
 * cnt holds |ATV|^{k'} for every ATV.  Writes up to cap candidates to out
 * (in frame order, then tuple order) and returns how many there are.  The
 * enumeration stops once more than cap+limit_extra candidates were seen;
 * limit_extra < 0 means never stop. */
/* Algorithm 4 on frame j alone.  Writes up to cap candidates to out, counts
 * every candidate of the frame into *n_out (which holds the candidates of
 * the frames before, so the stop rule sees the running total), and returns 1
 * if the enumeration stopped because *n_out exceeded cap + limit_extra
 * (limit_extra < 0: never).  out and cap are relative to this frame. */
static int restore_frame(const oracle_state *st, const uint32_t *cnt, uint32_t j, uint32_t *out, int64_t cap,
                         int64_t *n_out, int64_t base, int64_t limit)
{
    uint32_t r = st->p.r, cols = 1u << st->p.c;
    uint32_t T = oracle_threshold(st);
    uint32_t *sa[32];
    uint32_t nsa[32], val[32], msk[32], idx[32];
    int stop = 0, empty = 0;
    for (uint32_t i = 0; i < r; i++)
        sa[i] = (uint32_t *)malloc(sizeof(uint32_t) * cols);
    /* SA(i, j): super ATVs of row i in frame j, by column index. */
    for (uint32_t i = 0; i < r; i++) {
        nsa[i] = 0;
        for (uint32_t x = 0; x < cols; x++)
            if (cnt[(size_t)i * st->E + (((size_t)j << st->p.c) | x)] >= T)
                sa[i][nsa[i]++] = x;
        if (nsa[i] == 0)
            empty = 1;
    }
    if (!empty) {
        for (uint32_t i = 0; i < r; i++)
            idx[i] = 0;
        for (;;) {
            for (uint32_t i = 0; i < r; i++)
                place(st, i, sa[i][idx[i]], &val[i], &msk[i]);
            int ok = 1;
            for (uint32_t i = 0; i < r && ok; i++) {
                uint32_t i2 = (i + 1) % r;
                uint32_t dup = msk[i] & msk[i2];
                if (((val[i] ^ val[i2]) & dup) != 0)
                    ok = 0;
            }
            if (ok) {
                uint32_t L = 0;
                for (uint32_t i = 0; i < r; i++)
                    L |= val[i];
                uint32_t y = (uint32_t)(((uint64_t)L << st->p.u) | j);
                int64_t k = *n_out - base;
                if (k < cap)
                    out[k] = oracle_unmangle(st, y);
                (*n_out)++;
                if (limit >= 0 && *n_out > limit) {
                    stop = 1;
                    break;
                }
            }
            /* next tuple (odometer over the r rows) */
            uint32_t i = r;
            int wrapped = 0;
            while (i > 0) {
                i--;
                if (++idx[i] < nsa[i])
                    break;
                idx[i] = 0;
                if (i == 0)
                    wrapped = 1;
            }
            if (wrapped)
                break;
        }
    }
    for (uint32_t i = 0; i < r; i++)
        free(sa[i]);
    return stop;
}

int64_t oracle_restore(const oracle_state *st, const uint32_t *cnt, uint32_t *out, int64_t cap,
                       int64_t limit_extra)
{
    uint32_t nf = 1u << st->p.u;
    int64_t n_out = 0;
    int64_t limit = limit_extra >= 0 ? cap + limit_extra : -1;
    for (uint32_t j = 0; j < nf; j++) {
        int64_t base = n_out;
        int64_t room = cap > base ? cap - base : 0;
        if (restore_frame(st, cnt, j, out + (base < cap ? base : cap), room, &n_out, base, limit))
            break;
    }
    return n_out;
}

/* Algorithm 5 (NAT): the number of AT indices i that are active in all r
 * ATVs of RRH(aip). */
uint32_t oracle_nat(const oracle_state *st, uint32_t aip, uint32_t kp)
{
    uint32_t x[32], z;
    oracle_rrh(st, aip, x, &z);
    uint32_t nat = 0;
    for (uint32_t h = 0; h < st->p.g; h++) {
        int all = 1;
        for (uint32_t i = 0; i < st->p.r; i++) {
            if (!oracle_active(st, i, (z << st->p.c) | x[i], h, kp)) {
                all = 0;
                break;
            }
        }
        nat += (uint32_t)all;
    }
    return nat;
}

/* UP of frame j (Sec. 4.3): the product over rows of
 * P_{i,j} = |AAT(k',i,j)| / (g * 2^c). */
double oracle_up(const oracle_state *st, const uint64_t *aat, uint32_t j)
{
    uint32_t nf = 1u << st->p.u;
    double denom = (double)st->p.g * (double)(1u << st->p.c);
    double up = 1.0;
    for (uint32_t i = 0; i < st->p.r; i++)
        up *= (double)aat[(size_t)i * nf + j] / denom;
    return up;
}

/* Eq. 4: n = -g * ln((g - NAT) / (g * (1 - UP))).  Readings at the edges of
 * its domain: NAT = g (or UP = 1) gives +infinity (saturated); a ratio of 1
 * or more (NAT <= g*UP) gives 0.  With UP = 0 this is Eq. 2 with |ATV| =
 * NAT. */
double oracle_eq4(uint32_t g, uint32_t nat, double up)
{
    if (nat >= g || up >= 1.0)
        return INFINITY;
    double num = (double)(g - nat);
    double den = (double)g * (1.0 - up);
    double ratio = num / den;
    if (ratio >= 1.0)
        return 0.0;
    return -(double)g * log(ratio);
}

/* Eq. 2: n = -g * ln((g - |ATV|) / g), Eq. 1 with g0 = g - |ATV| zero bits. */
double oracle_eq2(uint32_t g, uint32_t cnt)
{
    if (cnt >= g)
        return INFINITY;
    return -(double)g * log((double)(g - cnt) / (double)g);
}

/* Cardinality estimate of one host at the end of the open slice (Sec. 4.3):
 * NAT by Algorithm 5, UP of its frame, Eq. 4. */
double oracle_estimate(const oracle_state *st, const uint64_t *aat, uint32_t aip, uint32_t kp,
                       uint32_t *nat_out)
{
    uint32_t x[32], z;
    oracle_rrh(st, aip, x, &z);
    uint32_t nat = oracle_nat(st, aip, kp);
    if (nat_out)
        *nat_out = nat;
    return oracle_eq4(st->p.g, nat, oracle_up(st, aat, z));
}

/* ------------------------------------------------------ all host cores */

/* The same functions run on several threads, for the timed CPU baseline:
 * the pool is split by (row, frame range), so no two threads write the same
 * AT and no atomics are needed.  Each result equals the single-thread call's
 * (the host tests compare them). */

#include <pthread.h>
#include <unistd.h>

int oracle_cores(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n < 1 ? 1 : (int)n;
}

typedef struct {
    oracle_state *st;
    const uint32_t *pairs;
    uint64_t lo, hi;        /* pair range (hash pass) */
    uint32_t *z, *x, *h;    /* per pair: frame, r columns, BH */
    uint32_t tid, nthreads; /* this thread's (row, frame) cells: every nthreads-th */
    uint64_t n;
    uint32_t kp;
    const uint32_t *cnt;
    uint32_t *cnt_out;
    const uint64_t *aat;
    const uint32_t *aips;
    double *est;
    uint32_t *nat;
    uint32_t *frame_out;
    int64_t frame_cap;
    int64_t *frame_counts;
} mt_job;

typedef void *(*mt_fn)(void *);

static void run_threads(mt_fn fn, mt_job *jobs, int nthreads)
{
    pthread_t th[256];
    for (int t = 1; t < nthreads; t++)
        pthread_create(&th[t], NULL, fn, &jobs[t]);
    fn(&jobs[0]);
    for (int t = 1; t < nthreads; t++)
        pthread_join(th[t], NULL);
}

static int clamp_threads(int nthreads)
{
    if (nthreads < 1)
        nthreads = oracle_cores();
    return nthreads > 256 ? 256 : nthreads;
}

/* Hash pass of Algorithm 3: RRH(aip) and BH(bip) of a range of pairs. */
static void *ingest_hash(void *arg)
{
    mt_job *j = (mt_job *)arg;
    uint32_t r = j->st->p.r, xx[32];
    for (uint64_t q = j->lo; q < j->hi; q++) {
        oracle_rrh(j->st, j->pairs[2 * q], xx, &j->z[q]);
        for (uint32_t i = 0; i < r; i++)
            j->x[q * r + i] = xx[i];
        j->h[q] = oracle_bh(j->st, j->pairs[2 * q + 1]);
    }
    return NULL;
}

/* Set pass of Algorithm 3: the ATs of this thread's (row, frame) cells. */
static void *ingest_set(void *arg)
{
    mt_job *j = (mt_job *)arg;
    oracle_state *st = j->st;
    uint32_t r = st->p.r, nf = 1u << st->p.u;
    for (uint64_t q = 0; q < j->n; q++) {
        uint32_t z = j->z[q], h = j->h[q];
        for (uint32_t i = 0; i < r; i++) {
            if ((i * nf + z) % j->nthreads != j->tid)
                continue;
            uint32_t est = (z << st->p.c) | j->x[q * r + i];
            uint32_t v = st->p.mode == 1 ? st->p.k : oracle_act(st, h);
            st->at[at_index(st, i, est, h)] = (uint8_t)v;
        }
    }
    return NULL;
}

/* oracle_ingest on nthreads threads (<= 0: every core), in chunks of pairs. */
void oracle_ingest_mt(oracle_state *st, const uint32_t *pairs, uint64_t n, int nthreads)
{
    nthreads = clamp_threads(nthreads);
    const uint64_t chunk = 1ull << 22;
    uint32_t r = st->p.r;
    uint32_t *z = (uint32_t *)malloc(sizeof(uint32_t) * chunk);
    uint32_t *x = (uint32_t *)malloc(sizeof(uint32_t) * chunk * r);
    uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * chunk);
    mt_job jobs[256];
    for (uint64_t c0 = 0; c0 < n; c0 += chunk) {
        uint64_t m = n - c0 < chunk ? n - c0 : chunk;
        for (int t = 0; t < nthreads; t++) {
            memset(&jobs[t], 0, sizeof(mt_job));
            jobs[t].st = st;
            jobs[t].pairs = pairs + 2 * c0;
            jobs[t].lo = m * (uint64_t)t / (uint64_t)nthreads;
            jobs[t].hi = m * (uint64_t)(t + 1) / (uint64_t)nthreads;
            jobs[t].z = z;
            jobs[t].x = x;
            jobs[t].h = h;
            jobs[t].tid = (uint32_t)t;
            jobs[t].nthreads = (uint32_t)nthreads;
            jobs[t].n = m;
        }
        run_threads(ingest_hash, jobs, nthreads);
        run_threads(ingest_set, jobs, nthreads);
    }
    free(z);
    free(x);
    free(h);
}

/* ATV ranges of (row, ATV) pairs: thread t takes ATVs [lo, hi) of the r*E. */
static void *advance_range(void *arg)
{
    mt_job *j = (mt_job *)arg;
    oracle_state *st = j->st;
    uint32_t k = st->p.k, g = st->p.g;
    for (uint64_t a = j->lo; a < j->hi; a++) {
        uint8_t *at = st->at + a * g;
        for (uint32_t hh = 0; hh < g; hh++) {
            if (st->p.mode == 1) {
                if (at[hh] != 0)
                    at[hh] -= 1;
            } else {
                at[hh] = (uint8_t)oracle_preserve_at(at[hh], oracle_act(st, hh), k);
            }
        }
    }
    return NULL;
}

/* oracle_advance on nthreads threads: the slice advances once, then each
 * thread applies Algorithm 2 (or the ACE decrement) to its ATVs. */
void oracle_advance_mt(oracle_state *st, int nthreads)
{
    nthreads = clamp_threads(nthreads);
    uint64_t total = (uint64_t)st->p.r * st->E;
    mt_job jobs[256];
    st->t += 1;
    for (int t = 0; t < nthreads; t++) {
        memset(&jobs[t], 0, sizeof(mt_job));
        jobs[t].st = st;
        jobs[t].lo = total * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = total * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    run_threads(advance_range, jobs, nthreads);
}

static void *counts_range(void *arg)
{
    mt_job *j = (mt_job *)arg;
    const oracle_state *st = j->st;
    for (uint64_t a = j->lo; a < j->hi; a++) {
        uint32_t row = (uint32_t)(a / st->E), e = (uint32_t)(a % st->E), n = 0;
        for (uint32_t hh = 0; hh < st->p.g; hh++)
            n += (uint32_t)oracle_active(st, row, e, hh, j->kp);
        j->cnt_out[a] = n;
    }
    return NULL;
}

/* oracle_counts on nthreads threads (ATV ranges). */
void oracle_counts_mt(oracle_state *st, uint32_t kp, uint32_t *cnt, int nthreads)
{
    nthreads = clamp_threads(nthreads);
    uint64_t total = (uint64_t)st->p.r * st->E;
    mt_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        memset(&jobs[t], 0, sizeof(mt_job));
        jobs[t].st = st;
        jobs[t].kp = kp;
        jobs[t].cnt_out = cnt;
        jobs[t].lo = total * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = total * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    run_threads(counts_range, jobs, nthreads);
}

static void *restore_frames(void *arg)
{
    mt_job *j = (mt_job *)arg;
    uint32_t nf = 1u << j->st->p.u;
    for (uint32_t f = j->tid; f < nf; f += j->nthreads) {
        int64_t n = 0;
        restore_frame(j->st, j->cnt, f, j->frame_out + (size_t)f * (size_t)j->frame_cap, j->frame_cap, &n, 0, -1);
        j->frame_counts[f] = n;
    }
    return NULL;
}

/* oracle_restore (no stop rule) with the frames spread over threads: every
 * frame's candidates (up to frame_cap each) are concatenated in frame order,
 * which is the single-thread order.  Returns the total count; out receives
 * the first cap. */
int64_t oracle_restore_mt(oracle_state *st, const uint32_t *cnt, uint32_t *out, int64_t cap, int64_t frame_cap,
                          int nthreads)
{
    nthreads = clamp_threads(nthreads);
    uint32_t nf = 1u << st->p.u;
    uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nf * (size_t)(frame_cap > 0 ? frame_cap : 1));
    int64_t *fn = (int64_t *)calloc(nf, sizeof(int64_t));
    mt_job jobs[256];
    int nt = nthreads < (int)nf ? nthreads : (int)nf;
    for (int t = 0; t < nt; t++) {
        memset(&jobs[t], 0, sizeof(mt_job));
        jobs[t].st = st;
        jobs[t].cnt = cnt;
        jobs[t].tid = (uint32_t)t;
        jobs[t].nthreads = (uint32_t)nt;
        jobs[t].frame_out = buf;
        jobs[t].frame_cap = frame_cap;
        jobs[t].frame_counts = fn;
    }
    run_threads(restore_frames, jobs, nt);
    int64_t n = 0;
    for (uint32_t f = 0; f < nf; f++) {
        int64_t m = fn[f] < frame_cap ? fn[f] : frame_cap;
        for (int64_t i = 0; i < m; i++)
            if (n + i < cap)
                out[n + i] = buf[(size_t)f * (size_t)frame_cap + (size_t)i];
        n += fn[f];
    }
    free(buf);
    free(fn);
    return n;
}

static void *estimate_range(void *arg)
{
    mt_job *j = (mt_job *)arg;
    for (uint64_t q = j->lo; q < j->hi; q++)
        j->est[q] = oracle_estimate(j->st, j->aat, j->aips[q], j->kp, &j->nat[q]);
    return NULL;
}

/* oracle_estimate of n hosts on nthreads threads. */
void oracle_estimate_mt(oracle_state *st, const uint64_t *aat, const uint32_t *aips, uint64_t n, uint32_t kp,
                        double *est, uint32_t *nat, int nthreads)
{
    nthreads = clamp_threads(nthreads);
    mt_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        memset(&jobs[t], 0, sizeof(mt_job));
        jobs[t].st = st;
        jobs[t].aat = aat;
        jobs[t].aips = aips;
        jobs[t].kp = kp;
        jobs[t].est = est;
        jobs[t].nat = nat;
        jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    run_threads(estimate_range, jobs, nthreads);
}
