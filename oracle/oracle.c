/*
 * FP64 CPU oracle for cascade-hashing feature matching.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file: only tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference legs of bench.py use it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * It is the plain, slow, step-by-step statement of the method of the paper
 * "Efficient Feature Matching for UAV Images based on Compact GPU Data
 * Scheduling", Sec. 2.3.1 (cascade hashing, steps (1)-(4), default parameters
 * L = 6, m = 8, n = 128, K = 8), with the readings listed below where the paper
 * is silent:
 *
 *  R1 hash family: random hyperplanes through the centred origin; weights
 *     W[k][h] i.i.d. N(0,1).  Columns 0 .. L*m-1 are the coarse bucket bits
 *     (table t uses columns t*m .. t*m+m-1), columns L*m .. L*m+nbits-1 the
 *     fine code.  Coarse and fine projections are independent.
 *  R2 weights come from one splitmix64 stream seeded with `seed`; each pair
 *     of outputs (r1, r2) gives u1 = ((r1>>11)+1)*2^-53 in (0,1],
 *     u2 = (r2>>11)*2^-53 in [0,1) and the Box-Muller pair
 *     z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2),
 *     filled in row-major order W[k][h] and rounded to float32.
 *  R3 centring: mu = (sum of all descriptors of the index) / N_total; the
 *     sums are exact integers.
 *  R4 a bit is 1 iff its projection s > 0 (strict).  Key bit b of table t is
 *     projection t*m+b (LSB first); code bit b is word b/32, bit b%32.
 *  R5 candidates of query p are the set union over the L tables of the
 *     database image's points in p's bucket (duplicates removed).
 *  R6 ranking by (Hamming distance, database index) ascending; the first
 *     min(K, |C|) are kept.
 *  R7 distances are Euclidean on the raw uint8 descriptors; q1, q2 are the
 *     first two kept candidates by (d^2, index).
 *  R8 ratio test dis(q1) < dis(q2) * t_r with t_r = num/den, evaluated
 *     exactly as den^2 * d1^2 < num^2 * d2^2.  Fewer than 2 candidates: no
 *     match.
 *  R9 a projection is "marginal" when |s| < 1e-4 * ||x - mu||_2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_D 128

/* ---- R2: splitmix64 (Steele, Lea & Flood, OOPSLA 2014) ------------------ */
static uint64_t orc_splitmix64(uint64_t* state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_first(uint64_t seed) { uint64_t s = seed; return orc_splitmix64(&s); }

/* Projection matrix W[128][P], P = L*m + nbits (R1, R2). */
void orc_weights(uint64_t seed, int32_t P, float* W) {
    uint64_t state = seed;
    const int64_t total = (int64_t)ORC_D * P;
    for (int64_t e = 0; e < total; e += 2) {
        uint64_t r1 = orc_splitmix64(&state);
        uint64_t r2 = orc_splitmix64(&state);
        double u1 = (double)((r1 >> 11) + 1) * (1.0 / 9007199254740992.0);
        double u2 = (double)(r2 >> 11) * (1.0 / 9007199254740992.0);
        double rad = sqrt(-2.0 * log(u1));
        double ang = 2.0 * M_PI * u2;
        W[e] = (float)(rad * cos(ang));
        if (e + 1 < total) W[e + 1] = (float)(rad * sin(ang));
    }
}

/* ---- R3: centring statistics ------------------------------------------- */
void orc_col_sums(const uint8_t* desc, int64_t n, uint64_t* sums) {
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < ORC_D; k++) sums[k] += desc[i * ORC_D + k];
}

/* ---- Sec. 2.3.1 steps (1)-(2): project, take signs -------------------------
 * Input: centred vectors xc[n][128] (FP64).  Output per vector: the L bucket
 * keys, the nbits-bit code and (optionally) one marginal flag per projection. */
void orc_hash_centred(const double* xc, int64_t n, const float* W, int32_t L, int32_t m, int32_t nbits,
                      uint8_t* keys, uint32_t* code, uint8_t* marginal) {
    const int32_t P = L * m + nbits;
    const int32_t nw = nbits / 32;
    double* s = (double*)malloc(sizeof(double) * (size_t)P);
    for (int64_t i = 0; i < n; i++) {
        const double* x = xc + i * ORC_D;
        double norm2 = 0.0;
        for (int k = 0; k < ORC_D; k++) norm2 += x[k] * x[k];
        const double tol = 1e-4 * sqrt(norm2);
        for (int h = 0; h < P; h++) {
            double acc = 0.0;
            for (int k = 0; k < ORC_D; k++) acc += (double)W[(int64_t)k * P + h] * x[k];
            s[h] = acc;
            if (marginal) marginal[i * P + h] = (uint8_t)(fabs(acc) < tol);
        }
        for (int t = 0; t < L; t++) {
            uint32_t key = 0;
            for (int b = 0; b < m; b++)
                if (s[t * m + b] > 0.0) key |= 1u << b;
            keys[i * L + t] = (uint8_t)key;
        }
        for (int w = 0; w < nw; w++) code[i * nw + w] = 0;
        for (int b = 0; b < nbits; b++)
            if (s[L * m + b] > 0.0) code[i * nw + b / 32] |= 1u << (b % 32);
    }
    free(s);
}

/* Raw descriptors: centre with mu (R3), then hash. */
void orc_hash(const uint8_t* desc, int64_t n, const double* mu, const float* W, int32_t L, int32_t m,
              int32_t nbits, uint8_t* keys, uint32_t* code, uint8_t* marginal) {
    double xc[ORC_D];
    const int32_t P = L * m + nbits;
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < ORC_D; k++) xc[k] = (double)desc[i * ORC_D + k] - mu[k];
        orc_hash_centred(xc, 1, W, L, m, nbits, keys + i * L, code + i * (nbits / 32),
                         marginal ? marginal + i * P : NULL);
    }
}

/* ---- Sec. 2.3.1 step (1): one lookup table of 2^m buckets per hash set ------
 * off[t][b] .. off[t][b+1] index idx[t][...], which lists the points of bucket b
 * in ascending order. */
void orc_buckets(const uint8_t* keys, int32_t n, int32_t L, int32_t m, int32_t* off, int32_t* idx) {
    const int32_t B = 1 << m;
    for (int t = 0; t < L; t++) {
        int32_t* o = off + (int64_t)t * (B + 1);
        for (int b = 0; b <= B; b++) o[b] = 0;
        for (int i = 0; i < n; i++) o[keys[(int64_t)i * L + t] + 1]++;
        for (int b = 0; b < B; b++) o[b + 1] += o[b];
        int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
        for (int b = 0; b < B; b++) fill[b] = o[b];
        for (int i = 0; i < n; i++) idx[(int64_t)t * n + fill[keys[(int64_t)i * L + t]]++] = i;
        free(fill);
    }
}

/* Hamming distance of two nbits-bit codes (Sec. 2.3.1 step (2)). */
static int orc_hamming(const uint32_t* a, const uint32_t* b, int32_t nw) {
    int h = 0;
    for (int w = 0; w < nw; w++) h += __builtin_popcount(a[w] ^ b[w]);
    return h;
}

/* Squared Euclidean distance of two raw descriptors (step (4), R7). */
static int64_t orc_dist2(const uint8_t* x, const uint8_t* y) {
    int64_t d = 0;
    for (int k = 0; k < ORC_D; k++) {
        int64_t e = (int64_t)x[k] - (int64_t)y[k];
        d += e * e;
    }
    return d;
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y);
}

typedef struct {
    int32_t n;
    const uint8_t* desc;     /* [n][128] */
    const uint8_t* keys;     /* [n][L] */
    const uint32_t* code;    /* [n][nbits/32] */
    const int32_t* off;      /* [L][2^m+1] */
    const int32_t* idx;      /* [L][n] */
} orc_image;

typedef struct {
    int32_t L, m, nbits, K;
    int32_t ratio_num, ratio_den;
} orc_params;

/* Match every query of I against database image J (Sec. 2.3.1 steps (1)-(4)).
 * Per query q: best_j[q] = index of q1 in J if the ratio test passes, else -1;
 * d1sq / d2sq = squared distances of q1 / q2 (UINT32_MAX where absent);
 * ncand[q] = |C(q)|; topk[q][0..K-1] = kept candidates in rank order, -1 padded.
 * Any output pointer except best_j may be NULL.  Returns the number of matches. */
int64_t orc_match_pair(const orc_image* I, const orc_image* J, const orc_params* p, int32_t q0, int32_t q1,
                       int32_t* best_j, uint32_t* d1sq, uint32_t* d2sq, int32_t* ncand, int32_t* topk) {
    const int32_t L = p->L, B = 1 << p->m, nw = p->nbits / 32, K = p->K;
    uint8_t* seen = (uint8_t*)calloc((size_t)(J->n > 0 ? J->n : 1), 1);
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(J->n > 0 ? J->n : 1));
    uint64_t* rank = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(J->n > 0 ? J->n : 1));
    int64_t matches = 0;
    for (int32_t q = q0; q < q1; q++) {
        const int32_t o = q - q0;
        /* step (1): union of the query's L buckets in J */
        int32_t nc = 0;
        for (int t = 0; t < L; t++) {
            const int b = I->keys[(int64_t)q * L + t];
            const int32_t* off = J->off + (int64_t)t * (B + 1);
            for (int32_t s = off[b]; s < off[b + 1]; s++) {
                int32_t j = J->idx[(int64_t)t * J->n + s];
                if (!seen[j]) { seen[j] = 1; cand[nc++] = j; }
            }
        }
        for (int32_t c = 0; c < nc; c++) seen[cand[c]] = 0;
        if (ncand) ncand[o] = nc;
        /* steps (2)-(3): rank by (Hamming, index) and keep the first K */
        for (int32_t c = 0; c < nc; c++) {
            uint64_t h = (uint64_t)orc_hamming(I->code + (int64_t)q * nw, J->code + (int64_t)cand[c] * nw, nw);
            rank[c] = (h << 32) | (uint64_t)cand[c];
        }
        qsort(rank, (size_t)nc, sizeof(uint64_t), cmp_u64);
        const int32_t kept = nc < K ? nc : K;
        if (topk)
            for (int32_t k = 0; k < K; k++) topk[(int64_t)o * K + k] = k < kept ? (int32_t)(rank[k] & 0xFFFFFFFFu) : -1;
        /* step (4): exact distances of the kept candidates, q1 and q2, ratio test */
        int64_t best1 = -1, best2 = -1;   /* candidate indices into J */
        int64_t e1 = 0, e2 = 0;           /* their squared distances */
        for (int32_t k = 0; k < kept; k++) {
            int64_t j = (int64_t)(rank[k] & 0xFFFFFFFFu);
            int64_t d = orc_dist2(I->desc + (int64_t)q * ORC_D, J->desc + j * ORC_D);
            if (best1 < 0 || d < e1 || (d == e1 && j < best1)) {
                best2 = best1; e2 = e1; best1 = j; e1 = d;
            } else if (best2 < 0 || d < e2 || (d == e2 && j < best2)) {
                best2 = j; e2 = d;
            }
        }
        int32_t out = -1;
        if (best2 >= 0) {
            const int64_t num = p->ratio_num, den = p->ratio_den;
            if (den * den * e1 < num * num * e2) out = (int32_t)best1;
        }
        best_j[o] = out;
        if (out >= 0) matches++;
        if (d1sq) d1sq[o] = best1 >= 0 ? (uint32_t)e1 : 0xFFFFFFFFu;
        if (d2sq) d2sq[o] = best2 >= 0 ? (uint32_t)e2 : 0xFFFFFFFFu;
    }
    free(seen); free(cand); free(rank);
    return matches;
}

/* Exhaustive nearest neighbours over all of J with the same ratio test (used by
 * the pin "cascade with one bucket and K = N_J equals brute force"). */
void orc_brute_nn(const uint8_t* descI, int32_t nI, const uint8_t* descJ, int32_t nJ, int32_t ratio_num,
                  int32_t ratio_den, int32_t* best_j, uint32_t* d1sq, uint32_t* d2sq) {
    for (int32_t q = 0; q < nI; q++) {
        int64_t b1 = -1, b2 = -1, e1 = 0, e2 = 0;
        for (int32_t j = 0; j < nJ; j++) {
            int64_t d = orc_dist2(descI + (int64_t)q * ORC_D, descJ + (int64_t)j * ORC_D);
            if (b1 < 0 || d < e1) { b2 = b1; e2 = e1; b1 = j; e1 = d; }
            else if (b2 < 0 || d < e2) { b2 = j; e2 = d; }
        }
        int32_t out = -1;
        if (b2 >= 0 && (int64_t)ratio_den * ratio_den * e1 < (int64_t)ratio_num * ratio_num * e2) out = (int32_t)b1;
        best_j[q] = out;
        d1sq[q] = b1 >= 0 ? (uint32_t)e1 : 0xFFFFFFFFu;
        d2sq[q] = b2 >= 0 ? (uint32_t)e2 : 0xFFFFFFFFu;
    }
}
