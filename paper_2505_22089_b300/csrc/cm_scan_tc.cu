// k_scan_tc: Hamming ranking and top-K (Sec. 2.3.1 steps (1)-(3)) with the
// Hamming distances computed on the tensor cores (thread mapping CM_ALGO_TC).
//
// Within one hash table, every query of the query image I that falls into
// bucket b meets every point of the database image J in the same bucket: the
// distances of a bucket form a dense n_I(b) x n_J(b) block.  With each code
// bit written as +1 / -1 in E4M3 (exact), the dot product of two codes is
// 128 - 2 h, an integer the FP32 accumulator holds exactly, so
//     h = (128 - x . y) / 2
// is the exact Hamming distance.  A bucket's codes and indices are contiguous
// in the bucket-sorted arrays, so every block is read with coalesced copies.
//
// One CTA takes a whole pair (all its queries, all tables); pairs are dealt
// round-robin.  Blocks are the bucket's query rows in tiles of 128 (M) times
// its database points in chunks of 128 (N), in the order (table, bucket,
// query tile, database chunk).  Roles:
//   warps 0-3    producers: cp.async the packed codes and indices of the block
//                R - 1 blocks ahead into a raw ring, then expand the codes into
//                E4M3 +-1 tiles (128-byte-swizzled K-major) through a byte
//                lookup table, into a stage ring;
//   warp 4       MMA issuer: tcgen05.mma kind::f8f6f4, M = 128, N = the
//                chunk's points rounded up to 16, K = 128 bits, into one of 4
//                TMEM accumulators;
//   warps 5-8    the epilogue (the 128 TMEM lanes = the tile's queries): for
//                every database chunk of a query tile it compares each
//                distance with the query's K-th kept key and inserts the
//                (h << 16 | j) keys that beat it; the top-K of the table stays
//                in registers across the tile's chunks and is stored as the
//                query's list for that table.  It waits on every stage and
//                accumulator phase in order (an mbarrier's parity only tells
//                apart consecutive phases).
// After the pair's last table the L lists of each query are merged (a key
// met in several tables is kept once) into its top-K, written to the
// hand-over the rerank launch reads (indices, squared norms, FP8 scales).
// Every wait is bounded; a wait that gives up sets the error flag and the
// roles run to the end without work, so every barrier is still met.
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_internal.h"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr int kScProdWarps = 4;
constexpr int kScProd = kScProdWarps * 32;
constexpr int kScMmaWarp = kScProdWarps;        // warp 4
constexpr int kScEpiWarp0 = kScProdWarps + 1;   // warps 5..8
constexpr int kScThreads = (kScProdWarps + 1 + 4) * 32;
constexpr int kScStages = 4;
constexpr int kScRaw = 6;                       // raw ring slots (blocks copied ahead)
constexpr int kScAcc = 4;                       // TMEM accumulators of 128 columns
constexpr int kScPolls = 1 << 24;
constexpr int kOffStride = 257;                 // bucket offsets per (table, image)
constexpr uint16_t kNoIdx = 0xFFFFu;

// stage: A tile | B tile | query ids | candidate ids | meta
constexpr uint32_t kTile = 128u * 128u;
constexpr uint32_t kStQ = 2 * kTile, kStC = kStQ + 256, kStMeta = kStC + 256;
constexpr uint32_t kStage = (kStMeta + 16 + 1023) / 1024 * 1024;
// raw slot: 256 codes (A rows 0-127, B rows 128-255) | A index words | B index words
constexpr uint32_t kRawIA = 256 * 16, kRawIB = kRawIA + 66 * 4, kRawSlot = kRawIB + 66 * 4;
// shared memory map (from the 1024-aligned base)
constexpr size_t kSmStages = 0;
constexpr size_t kSmRaw = kSmStages + (size_t)kScStages * kStage;
constexpr size_t kSmLut = kSmRaw + (size_t)kScRaw * kRawSlot;
constexpr size_t kSmPoff = kSmLut + 256 * 8;
constexpr size_t kSmEoff = kSmPoff + (size_t)kMaxL * 2 * kOffStride * 4;
constexpr size_t kSmBars = (kSmEoff + (size_t)kMaxL * 2 * kOffStride * 4 + 15) / 16 * 16;
constexpr size_t kSmTotal = kSmBars + 8 * (2 * kScStages + 2 * kScAcc);
constexpr size_t kSmAlloc = kSmTotal + 1024;
static_assert(kSmAlloc <= 227 * 1024, "shared memory");

__device__ __forceinline__ bool sc_wait(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
    if (*abort_flag) return false;
    for (int it = 0; it < kScPolls; it += 32) {
        if (tc::mbar_wait(mbar, parity, 32)) return true;
        if (*abort_flag) return false;
    }
    return false;
}

// decided once per warp, which continues only if every lane saw the phase; each
// lane waits itself, since the tcgen05 loads and shared-memory writes that
// follow are ordered after the phase only in a thread that observed it
__device__ __forceinline__ bool sc_warp_wait(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
    return __all_sync(0xFFFFFFFFu, sc_wait(mbar, parity, abort_flag));
}

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
}

// Keeps the K smallest keys in ascending order; a key already present is skipped.
template <int K>
__device__ __forceinline__ void sc_insert(uint32_t (&s)[K], uint32_t key) {
    bool dup = false;
#pragma unroll
    for (int i = 0; i < K; ++i) dup |= s[i] == key;
    if (dup) return;
#pragma unroll
    for (int i = K - 1; i > 0; --i) s[i] = max(s[i - 1], min(s[i], key));
    s[0] = min(s[0], key);
}

struct Blk {
    int t;
    int ia, na;    // query rows [ia, ia + na) of table t's bucket-sorted arrays of I
    int jb, nb;    // database rows [jb, jb + nb) of J's
    bool first, last;   // first / last database chunk of the query tile
};

// Walks the blocks of one pair from bucket offsets in shared memory:
// off[(t * 2 + 0) * 257 + b] for I, off[(t * 2 + 1) * 257 + b] for J.
struct Gen {
    const uint32_t* off;
    int L, B;
    int t = 0, b = -1, mi = 0, nc = 0, i0 = 0, ni = 0, j0 = 0, nj = 0;
    bool have = false;

    __device__ Gen(const uint32_t* o, int L_, int B_) : off(o), L(L_), B(B_) {}

    __device__ __forceinline__ bool next(Blk& o) {
        for (;;) {
            if (have) {
                if (nc < nj) {
                    o.t = t;
                    o.ia = i0 + mi;
                    o.na = min(128, ni - mi);
                    o.jb = j0 + nc;
                    o.nb = min(128, nj - nc);
                    o.first = nc == 0;
                    o.last = nc + 128 >= nj;
                    nc += 128;
                    return true;
                }
                mi += 128;
                nc = 0;
                if (mi < ni) continue;
                have = false;
            }
            if (++b >= B) {
                b = 0;
                if (++t >= L) {
                    t = L;
                    b = B;
                    return false;
                }
            }
            const uint32_t* oi = off + (t * 2) * kOffStride;
            const uint32_t* oj = oi + kOffStride;
            i0 = (int)oi[b];
            ni = (int)oi[b + 1] - i0;
            j0 = (int)oj[b];
            nj = (int)oj[b + 1] - j0;
            if (ni > 0 && nj > 0) {
                have = true;
                mi = 0;
                nc = 0;
            }
        }
    }
};

template <int K>
__global__ void __launch_bounds__(kScThreads, 1) k_scan_tc(MatchLaunch ml) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stages = sm + kSmStages;
    unsigned char* raw = sm + kSmRaw;
    const uint2* lut = reinterpret_cast<const uint2*>(sm + kSmLut);
    uint32_t* poff = reinterpret_cast<uint32_t*>(sm + kSmPoff);
    uint32_t* eoff = reinterpret_cast<uint32_t*>(sm + kSmEoff);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kSmBars);
    uint64_t* empty = full + kScStages;
    uint64_t* tfull = empty + kScStages;
    uint64_t* tempty = tfull + kScAcc;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int B = 1 << ml.m, L = ml.L;

    // byte v -> 8 E4M3 values: +1 (0x38) where bit k of v is set, -1 (0xB8) elsewhere
    for (int v = tid; v < 256; v += kScThreads) {
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lo |= (((v >> k) & 1) ? 0x38u : 0xB8u) << (8 * k);
            hi |= (((v >> (k + 4)) & 1) ? 0x38u : 0xB8u) << (8 * k);
        }
        reinterpret_cast<uint2*>(sm + kSmLut)[v] = make_uint2(lo, hi);
    }
    if (tid == 0) {
        for (int s = 0; s < kScStages; ++s) {
            tc::mbar_init(&full[s], kScProd);
            tc::mbar_init(&empty[s], 2);   // the MMAs have read the tiles; the epilogue has read the ids
        }
        for (int a = 0; a < kScAcc; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], 128);
        }
        s_abort = 0;
    }
    if (warp == kScMmaWarp) tc::tmem_alloc(&s_tmem, 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    auto give_up = [&]() {
        *abort_flag = 1;
        if (ml.err) atomicExch(ml.err, 1);
    };

    if (warp < kScProdWarps) {
        // ---------------- producers
        int k = 0;   // blocks handed to the MMA (all pairs)
        for (int p = blockIdx.x; p < ml.n_pairs; p += gridDim.x) {
            const DevPair P = ml.pairs[p];
            const DevImage I = ml.imgs[P.i], J = ml.imgs[P.j];
            named_sync(1, kScProd);   // the previous pair's walkers are done with poff
            for (int e = tid; e < L * (B + 1); e += kScProd) {
                const int t = e / (B + 1), b = e % (B + 1);
                poff[(t * 2) * kOffStride + b] = I.off[e];
                poff[(t * 2 + 1) * kOffStride + b] = J.off[e];
            }
            named_sync(1, kScProd);
            // raw copies of a block: codes (16 B each) and the 4-byte words holding its indices
            auto issue = [&](const Blk& bk, int slot) {
                if (bk.ia + bk.na > I.n || bk.jb + bk.nb > J.n) {   // offsets out of range: record, copy nothing
                    if (tid == 0 && ml.err) atomicExch(ml.err, 2);
                    return;
                }
                const uint32_t base = tc::smem_addr(raw + (size_t)slot * kRawSlot);
                const uint4* Ic = I.scode + (size_t)bk.t * I.n + bk.ia;
                const uint4* Jc = J.scode + (size_t)bk.t * J.n + bk.jb;
                for (int r = tid; r < bk.na + bk.nb; r += kScProd) {
                    if (r < bk.na) cp16(base + (uint32_t)r * 16u, Ic + r);
                    else cp16(base + (uint32_t)(128 + r - bk.na) * 16u, Jc + (r - bk.na));
                }
                const uint16_t* Ii = I.sidx + (size_t)bk.t * I.n + bk.ia;
                const uint16_t* Ji = J.sidx + (size_t)bk.t * J.n + bk.jb;
                const uintptr_t ia = reinterpret_cast<uintptr_t>(Ii) & ~(uintptr_t)3;
                const uintptr_t jb = reinterpret_cast<uintptr_t>(Ji) & ~(uintptr_t)3;
                const int wa = (int)((reinterpret_cast<uintptr_t>(Ii + bk.na) - ia + 3) / 4);
                const int wb = (int)((reinterpret_cast<uintptr_t>(Ji + bk.nb) - jb + 3) / 4);
                for (int w = tid; w < wa + wb; w += kScProd) {
                    if (w < wa) cp4(base + kRawIA + (uint32_t)w * 4u, reinterpret_cast<const void*>(ia + 4 * w));
                    else cp4(base + kRawIB + (uint32_t)(w - wa) * 4u, reinterpret_cast<const void*>(jb + 4 * (w - wa)));
                }
            };
            Gen gl(poff, L, B), ge(poff, L, B);
            Blk bl{};
            // prime: kScRaw - 1 blocks in flight (one commit group per block, empty groups at the end)
            for (int x = 0; x < kScRaw - 1; ++x) {
                if (gl.next(bl)) issue(bl, x);
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            Blk be{};
            int kk = 0;   // block of this pair
            while (ge.next(be)) {
                named_sync(1, kScProd);   // block kk - 1 is expanded: its raw slot may be refilled
                if (gl.next(bl)) issue(bl, (kk + kScRaw - 1) % kScRaw);
                asm volatile("cp.async.commit_group;" ::: "memory");
                asm volatile("cp.async.wait_group %0;" :: "n"(kScRaw - 1) : "memory");
                named_sync(1, kScProd);   // every producer's copies of block kk have landed
                const int s = k % kScStages;
                const uint32_t ph = (uint32_t)(k / kScStages) & 1u;
                const bool ok = sc_warp_wait(&empty[s], ph ^ 1u, abort_flag);
                unsigned char* st = stages + (size_t)s * kStage;
                const unsigned char* rs = raw + (size_t)(kk % kScRaw) * kRawSlot;
                if (ok) {
                    // expand: chunk e = 16 code bits of row e / 8 (A rows, then B rows)
                    for (int e = tid; e < (be.na + be.nb) * 8; e += kScProd) {
                        const int r = e >> 3, c = e & 7;
                        const bool isA = r < be.na;
                        const int rr = isA ? r : r - be.na;
                        const uint32_t w = *reinterpret_cast<const uint32_t*>(rs + (isA ? rr : 128 + rr) * 16 + (c >> 1) * 4);
                        const uint32_t bits = (w >> (16 * (c & 1))) & 0xFFFFu;
                        const uint2 lo = lut[bits & 0xFFu], hi = lut[bits >> 8];
                        *reinterpret_cast<uint4*>(st + (isA ? 0u : kTile) + rr * 128 + ((c ^ (rr & 7)) << 4)) =
                            make_uint4(lo.x, lo.y, hi.x, hi.y);
                    }
                    // ids: u16 element `par + x` of the copied words
                    const uint16_t* ra = reinterpret_cast<const uint16_t*>(rs + kRawIA);
                    const uint16_t* rb = reinterpret_cast<const uint16_t*>(rs + kRawIB);
                    const int pa = (int)((reinterpret_cast<uintptr_t>(I.sidx + (size_t)be.t * I.n + be.ia) >> 1) & 1);
                    const int pb = (int)((reinterpret_cast<uintptr_t>(J.sidx + (size_t)be.t * J.n + be.jb) >> 1) & 1);
                    uint16_t* qi = reinterpret_cast<uint16_t*>(st + kStQ);
                    uint16_t* ci = reinterpret_cast<uint16_t*>(st + kStC);
                    qi[tid] = tid < be.na ? ra[pa + tid] : (uint16_t)0;
                    ci[tid] = tid < be.nb ? rb[pb + tid] : kNoIdx;
                    if (tid == 0) reinterpret_cast<int*>(st + kStMeta)[0] = be.nb;
                } else {
                    give_up();
                }
                tc::fence_proxy_async();
                tc::mbar_arrive(&full[s]);
                ++k;
                ++kk;
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        // end of the sequence: a stage whose block has no database points
        const int s = k % kScStages;
        const uint32_t ph = (uint32_t)(k / kScStages) & 1u;
        if (sc_warp_wait(&empty[s], ph ^ 1u, abort_flag)) {
            if (tid == 0) reinterpret_cast<int*>(stages + (size_t)s * kStage + kStMeta)[0] = 0;
        } else {
            give_up();
            if (tid == 0) reinterpret_cast<int*>(stages + (size_t)s * kStage + kStMeta)[0] = 0;
        }
        tc::mbar_arrive(&full[s]);
    } else if (warp == kScMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            for (int k = 0;; ++k) {
                const int s = k % kScStages, a = k % kScAcc;
                const uint32_t ph = (uint32_t)(k / kScStages) & 1u, aph = (uint32_t)(k / kScAcc) & 1u;
                if (!sc_wait(&full[s], ph, abort_flag)) { give_up(); break; }
                const unsigned char* st = stages + (size_t)s * kStage;
                const int nb = reinterpret_cast<const int*>(st + kStMeta)[0];
                if (nb <= 0) break;
                if (!sc_wait(&tempty[a], aph ^ 1u, abort_flag)) { give_up(); break; }
                tc::fence_after();
                const uint32_t idesc = tc::idesc_e4m3(128, (nb + 15) & ~15);
                const uint32_t a0 = tc::smem_addr(st), b0 = a0 + kTile;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)   // K = 128 bits = 4 MMAs of 32 E4M3 values
                    tc::mma_f8f6f4(tmem + (uint32_t)(a * 128), tc::smem_desc_sw128(a0 + 32u * ks),
                                   tc::smem_desc_sw128(b0 + 32u * ks), idesc, ks != 0);
                tc::commit(&empty[s]);
                tc::commit(&tfull[a]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;        // TMEM lane = query row of the tile
        const int et = tid - kScEpiWarp0 * 32;    // 0..127
        uint32_t* lists = ml.lists + (size_t)blockIdx.x * (size_t)ml.max_ni * L * K;
        int k = 0;
        for (int p = blockIdx.x; p < ml.n_pairs; p += gridDim.x) {
            const DevPair P = ml.pairs[p];
            const DevImage I = ml.imgs[P.i], J = ml.imgs[P.j];
            named_sync(2, 128);   // the previous pair's offsets are no longer read
            for (int e = et; e < L * (B + 1); e += 128) {
                const int t = e / (B + 1), b = e % (B + 1);
                eoff[(t * 2) * kOffStride + b] = I.off[e];
                eoff[(t * 2 + 1) * kOffStride + b] = J.off[e];
            }
            named_sync(2, 128);
            Gen ge(eoff, L, B);
            Blk be{};
            uint32_t s[K];
#pragma unroll
            for (int v = 0; v < K; ++v) s[v] = kEmpty;
            int q = 0;
            while (ge.next(be)) {
                const int kb = k++;
                const int st_i = kb % kScStages, a = kb % kScAcc;
                const uint32_t ph = (uint32_t)(kb / kScStages) & 1u, aph = (uint32_t)(kb / kScAcc) & 1u;
                const bool valid = r < be.na;
                const unsigned char* st = stages + (size_t)st_i * kStage;
                if (be.first) {
#pragma unroll
                    for (int v = 0; v < K; ++v) s[v] = kEmpty;
                }
                // the stage stays ours until we release it: its ids are read in place
                bool ok = sc_warp_wait(&full[st_i], ph, abort_flag);
                ok = sc_warp_wait(&tfull[a], aph, abort_flag) && ok;
                if (!ok) give_up();
                tc::fence_after();
                if (be.first && valid && ok) q = reinterpret_cast<const uint16_t*>(st + kStQ)[r];
                const uint16_t* ci = reinterpret_cast<const uint16_t*>(st + kStC);
                const int N = (be.nb + 15) & ~15;
                for (int c0 = 0; c0 < N && ok; c0 += 16) {
                    uint32_t v[16];
                    tc::tmem_load16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(a * 128 + c0), v);
                    if (!valid) continue;
                    // h < h_K  <=>  dot > 128 - 2 h_K; equality is decided by the index, below
                    const float thr = 128.f - 2.f * (float)(s[K - 1] >> 16);
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float dot = __uint_as_float(v[c]);
                        if (dot >= thr) {
                            const uint32_t j = ci[c0 + c];
                            const uint32_t h = (uint32_t)__float2int_rn((128.f - dot) * 0.5f);
                            const uint32_t key = (h << 16) | j;
                            if (j != kNoIdx && key < s[K - 1]) sc_insert<K>(s, key);
                        }
                    }
                }
                tc::fence_before();
                tc::mbar_arrive(&tempty[a]);
                named_sync(2, 128);   // every epilogue thread is done with the stage's ids
                if (r == 0) tc::mbar_arrive(&empty[st_i]);
                if (be.last && valid && ok && q >= I.n) {   // an id out of range: record, store nothing
                    if (ml.err) atomicExch(ml.err, 2);
                } else if (be.last && valid && ok) {
                    uint4* dst = reinterpret_cast<uint4*>(lists + ((size_t)q * L + be.t) * K);
#pragma unroll
                    for (int v = 0; v < K / 4; ++v) dst[v] = make_uint4(s[4 * v], s[4 * v + 1], s[4 * v + 2], s[4 * v + 3]);
                }
            }
            named_sync(2, 128);   // every list of the pair is written
            // merge the L lists of each query (a table whose bucket had no database point left none)
            const bool fp8 = ml.rerank == CM_RERANK_FP8;
            for (int qq = et; qq < I.n; qq += 128) {
                uint32_t m[K];
#pragma unroll
                for (int v = 0; v < K; ++v) m[v] = kEmpty;
                const uint64_t kw = I.key[qq];
                for (int t = 0; t < L; ++t) {
                    const int bq = (int)((kw >> (8 * t)) & 0xFFu);
                    const uint32_t* oj = eoff + (t * 2 + 1) * kOffStride;
                    if (oj[bq + 1] == oj[bq]) continue;
                    const uint4* src = reinterpret_cast<const uint4*>(lists + ((size_t)qq * L + t) * K);
#pragma unroll
                    for (int v = 0; v < K / 4; ++v) {
                        const uint4 x = src[v];
                        const uint32_t kk4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (kk4[u] < m[K - 1]) sc_insert<K>(m, kk4[u]);
                    }
                }
                const int64_t row = P.row_off + qq;
#pragma unroll
                for (int v = 0; v < K; ++v) {
                    const int j = (int)(m[v] & 0xFFFFu);
                    if (m[v] != kEmpty && j >= J.n && ml.err) atomicExch(ml.err, 2);
                    const bool hv = m[v] != kEmpty && j < J.n;
                    ml.topk16[row * K + v] = hv ? (uint16_t)j : kNoIdx;
                    ml.hnorm[row * K + v] = hv ? __ldg(J.norm + j) : 0u;
                    if (fp8) ml.hscale[row * K + v] = hv ? __ldg(J.xscale + j) : 0.f;
                    if (ml.out.topk) ml.out.topk[row * K + v] = hv ? j : -1;
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == kScMmaWarp) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

template <int K>
cudaError_t launch_k(const MatchLaunch& m, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_scan_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmAlloc);
    if (e != cudaSuccess) return e;
    k_scan_tc<K><<<grid, kScThreads, kSmAlloc, s>>>(m);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_tc(const MatchLaunch& m, int grid, cudaStream_t s) {
    if (m.n_pairs == 0) return cudaSuccess;
    if (m.L > kMaxL || m.m > 8 || m.max_ni > 65535) return cudaErrorInvalidValue;
    const int g = m.n_pairs < grid ? m.n_pairs : grid;
    switch (m.K) {
        case 4: return launch_k<4>(m, g, s);
        case 8: return launch_k<8>(m, g, s);
        case 16: return launch_k<16>(m, g, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
