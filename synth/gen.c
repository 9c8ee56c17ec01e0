/*
 * Seeded synthetic workload generator (test and benchmark fixture).
 *
 * Produces uint8 128-d SIFT-like descriptors and keypoints for a set of images
 * that observe a shared "world" of tracks, so that neighbouring images share a
 * controlled fraction of descriptors as noisy copies.  It holds none of the
 * matching method's arithmetic: it only makes inputs.  Both the FP64 oracle
 * and the CUDA library consume what it writes.
 *
 * Recipe (one reading of "|N(0,1)| vectors L2-normalised and scaled to 0-255"):
 *   g_k = |N(0,1)|, u = g / ||g||_2, x_k = min(255, rint(255 * u_k)).
 *   A noisy observation of a track with base descriptor x is
 *   y_k = clip(rint(x_k + sigma * z_k), 0, 255), z_k ~ N(0,1).
 *
 * World model: a grid of cells_x * cells_y cells, each holding C tracks
 * numbered k = 0..C-1.  Image i covers a rectangle of cells and observes, in
 * every covered cell, the tracks k < q_i (so a smaller quota is a subset of a
 * larger one).  The remaining slots of the image are clutter (fresh
 * descriptors).  Observations and clutter are placed at random slots.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood 2014) run as a counter
 * stream keyed by (seed, tag, a, b).  Normal variates use a 2^16-entry
 * inverse-CDF table of the half-normal distribution plus a sign bit.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_D 128

typedef struct {
    uint64_t seed;
    int32_t cells_x, cells_y;
    int32_t tracks_per_cell;
    float img_w, img_h;     /* keypoint frame of every image, pixels */
    float kp_noise;         /* keypoint noise sigma, pixels */
} syn_world;

typedef struct {
    int32_t n;              /* descriptors in the image */
    int32_t cx0, cy0, cx1, cy1;  /* covered cells [cx0,cx1) x [cy0,cy1) */
    int32_t quota;          /* tracks observed per covered cell */
    float sigma;            /* descriptor noise of this image's observations */
    float A[6];             /* world (cell units) -> pixel affine map: u = A0 x + A1 y + A2, v = A3 x + A4 y + A5 */
} syn_image;

/* ---- splitmix64 counter streams ---------------------------------------- */
static inline uint64_t sm_next(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t sm_key(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b) {
    uint64_t s = sm_mix(seed + 0x632BE59BD9B4E019ull);
    s = sm_mix(s ^ (tag * 0x9E3779B97F4A7C15ull));
    s = sm_mix(s ^ (a + 0xD1B54A32D192ED03ull));
    s = sm_mix(s ^ (b * 0x8CB92BA72F3D8DD7ull + 1));
    return s;
}

enum { TAG_BASE = 1, TAG_NOISE = 2, TAG_CLUTTER = 3, TAG_PERM = 4, TAG_POS = 5, TAG_KP = 6 };

/* ---- half-normal inverse-CDF table ------------------------------------- */
static float g_hn[65536];
static pthread_once_t g_hn_once = PTHREAD_ONCE_INIT;

static void hn_init(void) {
    /* T[k] = sqrt(2) * erfinv((k + 0.5) / 65536), solved by bisection on erf. */
    for (int k = 0; k < 65536; k++) {
        double p = (k + 0.5) / 65536.0;
        double lo = 0.0, hi = 6.0;
        for (int it = 0; it < 80; it++) {
            double mid = 0.5 * (lo + hi);
            if (erf(mid) < p) lo = mid; else hi = mid;
        }
        g_hn[k] = (float)(M_SQRT2 * 0.5 * (lo + hi));
    }
}

static inline float half_normal(uint32_t r16) { return g_hn[r16 & 0xFFFF]; }
static inline float normal(uint32_t r32) {
    float v = g_hn[r32 & 0xFFFF];
    return (r32 & 0x80000000u) ? -v : v;
}

static void base_descriptor(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint8_t* out) {
    uint64_t s = sm_key(seed, tag, a, b);
    float g[SYN_D];
    double ss = 0.0;
    for (int k = 0; k < SYN_D; k += 4) {
        uint64_t r = sm_next(&s);
        for (int u = 0; u < 4; u++) {
            float v = half_normal((uint32_t)(r >> (16 * u)));
            g[k + u] = v;
            ss += (double)v * v;
        }
    }
    double inv = ss > 0 ? 255.0 / sqrt(ss) : 0.0;
    for (int k = 0; k < SYN_D; k++) {
        double v = rint(g[k] * inv);
        out[k] = (uint8_t)(v > 255.0 ? 255.0 : v);
    }
}

static void noisy_copy(uint64_t* s, float sigma, const uint8_t* x, uint8_t* y) {
    for (int k = 0; k < SYN_D; k += 2) {
        uint64_t r = sm_next(s);
        for (int u = 0; u < 2; u++) {
            double v = rint((double)x[k + u] + (double)sigma * normal((uint32_t)(r >> (32 * u))));
            y[k + u] = (uint8_t)(v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v));
        }
    }
}

static inline double unif(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Generate image `i`: descriptors [n][128], keypoints [n][2], track id per slot (-1 = clutter). */
static void gen_image(const syn_world* w, const syn_image* im, int64_t i,
                      uint8_t* desc, float* kp, int64_t* track) {
    const int n = im->n;
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int s = 0; s < n; s++) perm[s] = s;
    uint64_t ps = sm_key(w->seed, TAG_PERM, (uint64_t)i, 0);
    for (int s = n - 1; s > 0; s--) {            /* Fisher-Yates */
        int r = (int)(sm_next(&ps) % (uint64_t)(s + 1));
        int t = perm[s]; perm[s] = perm[r]; perm[r] = t;
    }
    int used = 0;
    uint8_t base[SYN_D];
    for (int cy = im->cy0; cy < im->cy1 && used < n; cy++) {
        for (int cx = im->cx0; cx < im->cx1 && used < n; cx++) {
            for (int k = 0; k < im->quota && used < n; k++) {
                int64_t tau = ((int64_t)cy * w->cells_x + cx) * w->tracks_per_cell + k;
                int slot = perm[used++];
                uint8_t* y = desc + (size_t)slot * SYN_D;
                base_descriptor(w->seed, TAG_BASE, (uint64_t)tau, 0, base);
                uint64_t ns = sm_key(w->seed, TAG_NOISE, (uint64_t)i, (uint64_t)tau);
                if (im->sigma > 0.f) noisy_copy(&ns, im->sigma, base, y);
                else memcpy(y, base, SYN_D);
                uint64_t pp = sm_key(w->seed, TAG_POS, (uint64_t)tau, 0);
                double wx = cx + unif(sm_next(&pp)), wy = cy + unif(sm_next(&pp));
                uint64_t r = sm_next(&ns);
                double u = im->A[0] * wx + im->A[1] * wy + im->A[2] + w->kp_noise * normal((uint32_t)r);
                double v = im->A[3] * wx + im->A[4] * wy + im->A[5] + w->kp_noise * normal((uint32_t)(r >> 32));
                if (kp) { kp[2 * (size_t)slot] = (float)u; kp[2 * (size_t)slot + 1] = (float)v; }
                if (track) track[slot] = tau;
            }
        }
    }
    for (int s = used; s < n; s++) {
        int slot = perm[s];
        base_descriptor(w->seed, TAG_CLUTTER, (uint64_t)i, (uint64_t)slot, desc + (size_t)slot * SYN_D);
        uint64_t ks = sm_key(w->seed, TAG_KP, (uint64_t)i, (uint64_t)slot);
        if (kp) {
            kp[2 * (size_t)slot] = (float)(unif(sm_next(&ks)) * w->img_w);
            kp[2 * (size_t)slot + 1] = (float)(unif(sm_next(&ks)) * w->img_h);
        }
        if (track) track[slot] = -1;
    }
    free(perm);
}

typedef struct {
    const syn_world* w;
    const syn_image* ims;
    const int64_t* row_off;   /* first row of each image in the output */
    int64_t i0, i1;
    uint8_t* desc; float* kp; int64_t* track;
    int64_t next;             /* shared work counter */
    pthread_mutex_t mu;
} gen_job;

static void* gen_worker(void* arg) {
    gen_job* j = (gen_job*)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->i1) break;
        int64_t r = j->row_off[i] - j->row_off[j->i0];
        gen_image(j->w, &j->ims[i], i, j->desc + (size_t)r * SYN_D,
                  j->kp ? j->kp + 2 * (size_t)r : NULL, j->track ? j->track + r : NULL);
    }
    return NULL;
}

/* Generate images [i0, i1) into concatenated outputs (rows of image i0 first).
 * row_off[i] = first row of image i in the whole dataset.  kp / track may be NULL. */
int syn_generate(const syn_world* w, const syn_image* ims, const int64_t* row_off,
                 int64_t i0, int64_t i1, uint8_t* desc, float* kp, int64_t* track, int n_threads) {
    pthread_once(&g_hn_once, hn_init);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    gen_job j = {w, ims, row_off, i0, i1, desc, kp, track, i0, PTHREAD_MUTEX_INITIALIZER};
    pthread_t th[256];
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, gen_worker, &j);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* Half-normal table value, exposed for the fixture's own tests. */
float syn_half_normal(uint32_t k) { pthread_once(&g_hn_once, hn_init); return g_hn[k & 0xFFFF]; }
