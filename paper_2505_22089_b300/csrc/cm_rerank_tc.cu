// Tensor-core rerank (Sec. 2.3.1 step (4), BF16 and FP8 forms).
//
// k_xcopy writes, after hashing, each resident descriptor once more in the
// rerank's operand type: BF16 (exact for uint8, 256-byte rows) or E4M3 scaled
// by the row maximum / 448 (128-byte rows, scale kept per row).
//
// k_rerank_tc takes the top-K lists the scan kernel left in global memory.  A
// sub-tile holds QS = 128 / K queries of one pair: its A operand is their K
// candidate rows each (M = 128), its B operand their QS query rows (N = NB >= 16,
// padded).  One MMA chain (K = 128) gives every candidate's dot product with
// every query of the sub-tile, of which candidate row r needs column r / K.
// The kernel is persistent and warp-specialised, work items dealt
// round-robin (the launch shape per form is in RR below):
//   producers    16-byte cp.async copies of the A and B rows from the
//                row copies into a ring of shared-memory stages, in the
//                128-byte-swizzled K-major operand layout; each thread's copies
//                arrive on the stage's mbarrier as they land
//                (cp.async.mbarrier.arrive.noinc), so every stage of the ring
//                can be in flight and no thread waits for its own copies;
//   MMA issuer   one thread, a proxy fence after each stage's wait
//                (generic-proxy copies before async-proxy reads),
//                tcgen05.mma into one of ACC TMEM accumulators, commits that
//                free the stage and fill the accumulator;
//   epilogue     groups of 4 warps (each the 128 TMEM lanes), taking the
//                sub-tiles in turn: d^2 = |x|^2 + |y|^2 - 2 x.y,
//                q1 / q2 by (d^2, index) across the K lanes of a query, the
//                exact ratio test, outputs.
//   BF16: the dot is an exact integer in FP32, so d^2 is exact.
//   FP8:  the approximate d^2 picks q1, q2, which are re-scored exactly on
//         CUDA cores; a re-score that reverses their order is counted.
// Every wait is bounded; a wait that gives up sets the error flag and ends the
// kernel's loops.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdint>

#include "cm_internal.h"
#include "cm_ratio.cuh"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr int kRrSleeps = 1 << 20;
constexpr uint16_t kNoCand = 0xFFFFu;

template <int K, bool FP8>
struct RR {
    // Launch shape, both forms: two CTAs per SM (two MMA issuers; one issuing
    // thread's 8 MMAs per sub-tile bounded a CTA), 4 producer warps and one
    // epilogue group each.  Two epilogue groups per CTA do not fit the
    // register file twice: BF16 then needs fewer producers and lost, FP8
    // spilled and was no faster.
    static constexpr int CTAS = 2;                        // CTAs per SM
    static constexpr int PROD_WARPS = 4;
    static constexpr int PROD = PROD_WARPS * 32;          // producer threads
    static constexpr int MMA_WARP = PROD_WARPS;
    static constexpr int EPI_WARP0 = PROD_WARPS + 1;
    static constexpr int EPI = 1;                         // epilogue groups of 4 warps, taking sub-tiles in turn
    static constexpr int THREADS = (PROD_WARPS + 1 + 4 * EPI) * 32;
    static constexpr int QS = 128 / K;                    // queries per sub-tile
    static constexpr int NB = QS < 16 ? 16 : QS;          // B rows = MMA N
    static constexpr int HALVES = FP8 ? 1 : 2;            // 128-byte column blocks per row
    static constexpr uint32_t A_HALF = 128u * 128u;       // 128 rows x 128 bytes
    static constexpr uint32_t B_HALF = (uint32_t)NB * 128u;
    static constexpr uint32_t STAGE = HALVES * (A_HALF + B_HALF);
    static constexpr int STAGES_FIT = (int)((216u * 1024u / CTAS) / STAGE);
    static constexpr int STAGES = STAGES_FIT < 8 ? STAGES_FIT : 8;
    static constexpr int ACC_FIT = 256 / NB;
    static constexpr int ACC = ACC_FIT < 8 ? ACC_FIT : 8;  // a multiple of the epilogue groups, which take turns
    static constexpr int STEPS = FP8 ? 4 : 8;              // MMAs of 32 bytes of K each
    static constexpr int CPR = FP8 ? 8 : 16;               // 16-byte chunks per row copy
    // stages (1024-aligned) + barriers: full/empty per stage, full/empty per accumulator
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 8 * (2 * STAGES + 2 * ACC) + 64;
    static_assert(ACC % EPI == 0, "accumulators are dealt to the epilogue groups in turn");
    static_assert(STAGES >= 2, "stage ring");
    static_assert(256 * CTAS <= 512, "each CTA allocates 256 TMEM columns");
    static_assert(B_HALF % 1024 == 0, "B tile keeps 1024-byte alignment");
};

// A sub-tile: QS consecutive queries of one pair.  Sub-tile u is part u % per_item
// of work item u / per_item; CTA b takes u = b, b + grid, ..., so at any moment
// the CTAs work on neighbouring sub-tiles of the same one or two pairs and
// share the database rows they read in L2.
struct SubTile {
    int q0;        // first query (local row of image i)
    int nq;        // queries (<= QS); 0 = nothing to do
    int64_t row;   // output row of the first query
    // the pair's images: row copies, query norms / scales, raw rows (FP8 re-score)
    const unsigned char *ixq, *jxq;
    const uint32_t *inorm, *jnorm;
    const float *iscale, *jscale;
    const uint8_t *idesc, *jdesc;
    int n_j;       // rows of the database image
};

// Index of kept candidate e (flat [row][K] position) and, from the plan's
// hand-over or the bucket-major scan's key lists (Hamming << 16 | index; an
// empty key's low half is kNoCand as well), whether it exists.
__device__ __forceinline__ uint32_t cand_index(const MatchLaunch& ml, int64_t e) {
    return ml.topk16 ? (uint32_t)ml.topk16[e] : (ml.klists[e] & 0xFFFFu);
}

// Walks a CTA's increasing sequence of sub-tiles; the current pair's record is
// kept in registers and replaced only when the sequence crosses into a later
// pair.  The next pair's record is loaded at the previous crossing, so a
// crossing waits at most for the image records (IMG) and not for a chain of
// dependent loads; the MMA issuer needs no image record at all.
template <bool IMG>
struct Cursor {
    int pair = -1, item0 = 0, item_end = 0, n_i = 0;
    int64_t row_off = 0;
    const unsigned char *ixq = nullptr, *jxq = nullptr;
    const uint32_t *inorm = nullptr, *jnorm = nullptr;
    const float *iscale = nullptr, *jscale = nullptr;
    const uint8_t *idesc = nullptr, *jdesc = nullptr;
    int n_j = 0;
    DevPair nxt{};   // record of pair + 1
    // u = item * per_item + part, stepped without a division when u grows by the grid
    int last_u = -1, cur_item = 0, cur_part = 0, step_item = 0, step_part = 0;

    __device__ __forceinline__ SubTile at(const MatchLaunch& ml, int u, int per_item, int qs) {
        if (last_u >= 0 && u == last_u + (int)gridDim.x) {
            cur_item += step_item;
            cur_part += step_part;
            if (cur_part >= per_item) {
                cur_part -= per_item;
                ++cur_item;
            }
        } else {
            step_item = (int)gridDim.x / per_item;
            step_part = (int)gridDim.x % per_item;
            cur_item = u / per_item;
            cur_part = u % per_item;
        }
        last_u = u;
        const int item = cur_item;
        while (item >= item_end && pair + 1 < ml.n_pairs) {
            ++pair;
            const DevPair P = pair == 0 ? ml.pairs[0] : nxt;
            if (pair + 1 < ml.n_pairs) nxt = ml.pairs[pair + 1];   // used at the next crossing
            item0 = P.item0;
            item_end = P.item0 + P.nitems;
            row_off = P.row_off;
            n_i = P.ni;
            if (IMG) {
                const DevImage& I = ml.imgs[P.i];
                const DevImage& J = ml.imgs[P.j];
                ixq = static_cast<const unsigned char*>(I.xq);
                jxq = static_cast<const unsigned char*>(J.xq);
                n_j = J.n;
                inorm = I.norm;
                jnorm = J.norm;
                iscale = I.xscale;
                jscale = J.xscale;
                idesc = I.desc;
                jdesc = J.desc;
            }
        }
        SubTile t;
        t.q0 = (item - item0) * ml.S + cur_part * qs;
        t.nq = (item < item_end && t.q0 < n_i) ? min(qs, n_i - t.q0) : 0;
        t.row = row_off + t.q0;
        t.ixq = ixq;
        t.jxq = jxq;
        t.inorm = inorm;
        t.jnorm = jnorm;
        t.iscale = iscale;
        t.jscale = jscale;
        t.idesc = idesc;
        t.jdesc = jdesc;
        t.n_j = n_j;
        return t;
    }
};

// Bounded wait for an mbarrier phase that also gives up once another role
// aborted: sleeping try_waits of at most 2 us each, about 2 s in all.
__device__ __forceinline__ bool wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
    for (int it = 0; it < kRrSleeps; ++it) {
        if (tc::mbar_try_wait_sleep(mbar, parity, 2000)) return true;
        if (*abort_flag) return false;
    }
    return false;
}

// The same for a whole warp, which continues only if every lane saw the phase.
// Every lane waits on the barrier itself: a tcgen05.ld or a shared-memory
// write that must come after the phase is ordered after it only in a thread
// that observed the phase.  With lane 0 alone polling and passing its result
// on by shuffle, some builds read accumulators before the MMA had written them.
__device__ __forceinline__ bool warp_wait(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
    return __all_sync(0xFFFFFFFFu, wait_or_abort(mbar, parity, abort_flag));
}

__device__ __forceinline__ uint32_t exact_d2(const uint8_t* x, const uint8_t* y, int nb) {
    uint32_t acc = 0;
    for (int o = 0; o < nb; o += 16) {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(x + o));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(y + o));
        const uint32_t d0 = __vabsdiffu4(a.x, b.x), d1 = __vabsdiffu4(a.y, b.y);
        const uint32_t d2 = __vabsdiffu4(a.z, b.z), d3 = __vabsdiffu4(a.w, b.w);
        acc = __dp4a(d0, d0, acc);
        acc = __dp4a(d1, d1, acc);
        acc = __dp4a(d2, d2, acc);
        acc = __dp4a(d3, d3, acc);
    }
    return acc;
}

template <int K, bool FP8>
__global__ void __launch_bounds__(RR<K, FP8>::THREADS, RR<K, FP8>::CTAS) k_rerank_tc(MatchLaunch ml) {
    using C = RR<K, FP8>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)C::STAGES * C::STAGE);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;
    uint64_t* tempty = tfull + C::ACC;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ uint32_t s_stats[3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(&full[s], C::PROD);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < C::ACC; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], 128);
        }
        s_abort = 0;
        s_stats[0] = s_stats[1] = s_stats[2] = 0;
    }
    if (warp == C::MMA_WARP) tc::tmem_alloc(&s_tmem, 256);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;

    auto give_up = [&]() {
        *abort_flag = 1;
        if (ml.err) atomicExch(ml.err, 1);
    };
    const int per_item = ml.S / C::QS;
    const int n_sub = ml.n_items * per_item;
    // Every role walks the same sequence of non-empty sub-tiles, so the local
    // counter `it` (stage it % STAGES, accumulator it % ACC) agrees across roles.

    if (warp < C::PROD_WARPS) {
        // ---------------- producers.  Thread t copies the 16-byte chunk c = t % CPR of the
        // RPT consecutive A rows r0 = RPT * (t / CPR) .. r0 + RPT - 1 (the same chunk of
        // every row, so the swizzle term of each row is fixed at compile time up to c)
        // and of the B rows t / CPR + G q.  A warp's copies of one row index cover whole
        // rows (coalesced).
        constexpr int RPT = 128 * C::CPR / C::PROD;   // A rows per thread
        constexpr int G = C::PROD / C::CPR;            // threads per chunk column
        constexpr int NW = RPT / 2;                    // 32-bit words of RPT 16-bit indices
        // the RPT indices of a thread's rows are contiguous in the hand-over; one vector
        // load takes them when the sub-tile's first row keeps it aligned
        constexpr int VB = 2 * RPT < 16 ? 2 * RPT : 16;
        constexpr bool VEC = (2 * K) % VB == 0;
        static_assert(RPT % 2 == 0 && 128 % RPT == 0, "rows per producer thread");
        const int rb = FP8 ? 128 : 256;   // bytes per row copy
        const int c = tid % C::CPR, rg = tid / C::CPR;
        const int r0 = RPT * rg;
        const uint32_t cofs = (uint32_t)(c >> 3) * C::A_HALF;   // 128-byte column block of chunk c
        const uint32_t bofs = (uint32_t)(c >> 3) * C::B_HALF;
        const int c8 = c & 7;
        int it = 0;          // sub-tiles issued
        Cursor<true> cursor;
        bool ok = true;
        int u = blockIdx.x - (int)gridDim.x;
        // advances to the next non-empty sub-tile of this CTA's sequence
        auto next = [&](SubTile& t) -> bool {
            for (u += gridDim.x; u < n_sub; u += gridDim.x) {
                t = cursor.at(ml, u, per_item, C::QS);
                if (t.nq > 0) return true;
            }
            return false;
        };
        // candidate indices of the thread's rows, two per word (kNoCand: no candidate);
        // loaded one sub-tile before they are used
        auto idx_of = [&](const SubTile& t, uint32_t (&jw)[NW]) {
            const int64_t e0 = t.row * K + r0;
            if (VEC && ml.topk16 && (r0 + RPT - 1) / K < t.nq) {
                if constexpr (VB == 16) {
                    const uint4* p = reinterpret_cast<const uint4*>(ml.topk16 + e0);
#pragma unroll
                    for (int w = 0; w < NW / 4; ++w) {
                        const uint4 v = __ldg(p + w);
                        jw[4 * w] = v.x;
                        jw[4 * w + 1] = v.y;
                        jw[4 * w + 2] = v.z;
                        jw[4 * w + 3] = v.w;
                    }
                } else if constexpr (VB == 8) {
                    const uint2 v = __ldg(reinterpret_cast<const uint2*>(ml.topk16 + e0));
                    jw[0] = v.x;
                    jw[1] = v.y;
                } else {
                    jw[0] = __ldg(reinterpret_cast<const uint32_t*>(ml.topk16 + e0));
                }
                return;
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int ra = r0 + 2 * w, rc = ra + 1;
                const uint32_t lo = ra / K < t.nq ? cand_index(ml, e0 + 2 * w) : (uint32_t)kNoCand;
                const uint32_t hi = rc / K < t.nq ? cand_index(ml, e0 + 2 * w + 1) : (uint32_t)kNoCand;
                jw[w] = lo | (hi << 16);
            }
        };
        // copies sub-tile t into stage it % STAGES; the stage goes to the MMA once every
        // producer thread's copies into it have landed
        auto issue = [&](const SubTile& t, const uint32_t (&jw)[NW]) -> bool {
            const int s = it % C::STAGES;
            const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
            if (!warp_wait(&empty[s], ph ^ 1u, abort_flag)) return false;
            const uint32_t A = tc::smem_addr(ring + (size_t)s * C::STAGE) + cofs;
            const uint32_t B = tc::smem_addr(ring + (size_t)s * C::STAGE) + C::HALVES * C::A_HALF + bofs;
            const unsigned char* qrow = t.ixq + (size_t)t.q0 * rb + c * 16;   // a valid row for padding
            // an empty slot (kNoCand) copies the database image's last row, a real row whose
            // product the epilogue ignores; with no database row at all, the query row
            const unsigned char* jrow = t.n_j > 0 ? t.jxq + c * 16 : qrow;
            const uint32_t jmax = t.n_j > 0 ? (uint32_t)(t.n_j - 1) : 0u;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = r0 + q;
                const uint32_t j = (jw[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
                const uint32_t dst = A + (uint32_t)r * 128u + (uint32_t)((c8 ^ (r & 7)) << 4);
                const unsigned char* src = jrow + (size_t)min(j, jmax) * rb;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
            }
#pragma unroll
            for (int q = 0; q < (C::NB + G - 1) / G; ++q) {
                const int b = rg + G * q;
                if (b < C::NB) {
                    const uint32_t dst = B + (uint32_t)b * 128u + (uint32_t)((c8 ^ (b & 7)) << 4);
                    const unsigned char* src = qrow + (size_t)(b < t.nq ? b : 0) * rb;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
                }
            }
            // this thread's arrival on the stage, made when all its copies so far have landed
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(tc::smem_addr(&full[s]))
                         : "memory");
            ++it;
            return true;
        };
        // ping-pong between two register sets, so a prefetched index is never copied
        // (a copy would wait for the load)
        SubTile tA{}, tB{};
        uint32_t jA[NW], jB[NW];
        bool hA = next(tA), hB = false;
        if (hA) idx_of(tA, jA);
        while (hA) {
            hB = next(tB);
            if (hB) idx_of(tB, jB);
            if (!issue(tA, jA)) { ok = false; break; }
            if (!hB) break;
            hA = next(tA);
            if (hA) idx_of(tA, jA);
            if (!issue(tB, jB)) { ok = false; break; }
        }
        if (!ok) give_up();
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == C::MMA_WARP) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = FP8 ? tc::idesc_e4m3(128, C::NB) : tc::idesc_f16(128, C::NB, 1);
            int it = 0;
            Cursor<false> cursor;
            for (int u = blockIdx.x; u < n_sub; u += gridDim.x) {
                const SubTile t = cursor.at(ml, u, per_item, C::QS);
                if (t.nq <= 0) continue;
                const int s = it % C::STAGES, a = it % C::ACC;
                const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u, aph = (uint32_t)(it / C::ACC) & 1u;
                if (!wait_or_abort(&full[s], ph, abort_flag)) { give_up(); break; }
                if (!wait_or_abort(&tempty[a], aph ^ 1u, abort_flag)) { give_up(); break; }
                tc::fence_proxy_async();   // the producers' copies (generic proxy) before the MMA's reads
                tc::fence_after();
                const uint32_t a0 = tc::smem_addr(ring + (size_t)s * C::STAGE);
                const uint32_t b0 = a0 + C::HALVES * C::A_HALF;
#pragma unroll
                for (int ks = 0; ks < C::STEPS; ++ks) {
                    const uint32_t ah = a0 + (uint32_t)(ks >> 2) * C::A_HALF + (uint32_t)(ks & 3) * 32u;
                    const uint32_t bh = b0 + (uint32_t)(ks >> 2) * C::B_HALF + (uint32_t)(ks & 3) * 32u;
                    if (FP8)
                        tc::mma_f8f6f4(tmem + (uint32_t)(a * C::NB), tc::smem_desc_sw128(ah), tc::smem_desc_sw128(bh),
                                       idesc, ks != 0);
                    else
                        tc::mma_f16(tmem + (uint32_t)(a * C::NB), tc::smem_desc_sw128(ah), tc::smem_desc_sw128(bh),
                                    idesc, ks != 0);
                }
                tc::commit(&empty[s]);   // the stage may be refilled once these MMAs have read it
                tc::commit(&tfull[a]);   // the accumulator is complete
                ++it;
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: group g takes the sub-tiles with it % EPI == g
        const int g = (warp - C::EPI_WARP0) >> 2;
        const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31
        const int r = 32 * quarter + lane;          // candidate row of the A tile
        const int c = r / K, k = r % K;             // its query column and slot
        constexpr int W = 32 / K;                   // columns of this warp's 32 rows (W >= 2)
        static_assert(W == 2 || W == 4 || W == 8 || W == 16, "TMEM load width");
        const int col0 = 32 * quarter / K;          // the first of them
        uint32_t rechecks = 0, matches = 0, swaps = 0;
        // inputs of one sub-tile for this thread: all contiguous (hand-over written by the scan)
        struct In {
            uint32_t j, ny, nx;
            float sy, sx;
        };
        auto fetch = [&](const SubTile& t) {
            In v{kNoCand, 0u, 0u, 1.f, 1.f};
            if (c < t.nq) {
                const int64_t e = (t.row + c) * K + k;
                v.j = cand_index(ml, e);
                const bool hv = v.j != kNoCand;
                v.ny = ml.hnorm ? ml.hnorm[e] : (hv ? __ldg(t.jnorm + v.j) : 0u);
                v.nx = __ldg(t.inorm + t.q0 + c);
                if (FP8) {
                    v.sy = ml.hscale ? ml.hscale[e] : (hv ? __ldg(t.jscale + v.j) : 0.f);
                    v.sx = __ldg(t.iscale + t.q0 + c);
                }
            }
            return v;
        };
        int it = 0;          // position in the CTA's sequence of non-empty sub-tiles
        Cursor<true> cursor;
        int u = blockIdx.x - (int)gridDim.x;
        // advances to this group's next sub-tile (every EPI-th of the sequence)
        auto next = [&](SubTile& t, int& myit) -> bool {
            for (u += gridDim.x; u < n_sub; u += gridDim.x) {
                t = cursor.at(ml, u, per_item, C::QS);
                if (t.nq <= 0) continue;
                const int pos = it++;
                if (pos % C::EPI == g) {
                    myit = pos;
                    return true;
                }
            }
            return false;
        };
        auto process = [&](const SubTile& t, const In& v, int myit) -> bool {
            const int a = myit % C::ACC;
            const uint32_t aph = (uint32_t)(myit / C::ACC) & 1u;
            const bool qv = c < t.nq;
            const int qi = t.q0 + (qv ? c : 0);
            const bool hv = v.j != kNoCand;
            const int j = hv ? (int)v.j : 0;
            if (!warp_wait(&tfull[a], aph, abort_flag)) return false;
            tc::fence_after();
            uint32_t vv[W];
            tc::tmem_load<W>(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(a * C::NB + col0), vv);
            // column c = col0 + lane / K, picked by a binary tree of selects on the
            // bits of lane / K (the values stay in registers)
            const int sel = lane / K;
#pragma unroll
            for (int w = W / 2, bit = 1; w >= 1; w /= 2, bit *= 2)
#pragma unroll
                for (int q = 0; q < w; ++q) vv[q] = (sel & bit) ? vv[2 * q + 1] : vv[2 * q];
            const float dot = __uint_as_float(vv[0]);
            tc::fence_before();
            tc::mbar_arrive(&tempty[a]);   // this thread's lane of the accumulator is read

            uint64_t mine = ~0ull;
            if (hv) {
                if (!FP8) {
                    const uint32_t d2 = (uint32_t)((float)v.nx + (float)v.ny - 2.f * dot);   // exact: integers < 2^24
                    mine = ((uint64_t)d2 << 32) | (uint32_t)j;
                } else {
                    // each step rounded on its own (no contraction into an FMA), so the
                    // approximate distance, and with it the pick of q1 and q2 among near
                    // ties, does not depend on how a build schedules the expression
                    const float d2a = fmaxf(__fsub_rn(__fadd_rn((float)v.nx, (float)v.ny),
                                                      __fmul_rn(__fmul_rn(__fmul_rn(2.f, dot), v.sx), v.sy)),
                                            0.f);
                    mine = ((uint64_t)__float_as_uint(d2a) << 32) | (uint32_t)j;
                }
            }
            // q1, q2 over the K lanes of this query
            uint64_t m1 = mine;
#pragma unroll
            for (int o = K / 2; o > 0; o >>= 1) m1 = min(m1, __shfl_xor_sync(0xFFFFFFFFu, m1, o));
            uint64_t m2 = mine == m1 ? ~0ull : mine;
#pragma unroll
            for (int o = K / 2; o > 0; o >>= 1) m2 = min(m2, __shfl_xor_sync(0xFFFFFFFFu, m2, o));
            int j1 = m1 != ~0ull ? (int)(m1 & 0xFFFFu) : -1;
            int j2 = m2 != ~0ull ? (int)(m2 & 0xFFFFu) : -1;
            uint32_t d1 = j1 >= 0 ? (uint32_t)(m1 >> 32) : kEmpty;
            uint32_t d2 = j2 >= 0 ? (uint32_t)(m2 >> 32) : kEmpty;
            if (FP8) {
                // exact re-score of q1 and q2: half of the K lanes per row
                constexpr int LPR = K / 2 > 0 ? K / 2 : 1;
                constexpr int NBYTES = 128 / LPR;
                const int half = k / LPR, part = k % LPR;
                const int jr = half == 0 ? j1 : j2;
                uint32_t e = 0;
                if (qv && jr >= 0)
                    e = exact_d2(t.idesc + (size_t)qi * kDim + part * NBYTES,
                                 t.jdesc + (size_t)jr * kDim + part * NBYTES, NBYTES);
#pragma unroll
                for (int o = LPR / 2; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
                const int gbase = lane & ~(K - 1);
                const uint32_t e1 = __shfl_sync(0xFFFFFFFFu, e, gbase);
                const uint32_t e2 = __shfl_sync(0xFFFFFFFFu, e, gbase + LPR);
                d1 = j1 >= 0 ? e1 : kEmpty;
                d2 = j2 >= 0 ? e2 : kEmpty;
                if (j2 >= 0 && (d2 < d1 || (d2 == d1 && j2 < j1))) {   // the re-score reverses q1, q2
                    const uint32_t td = d1; d1 = d2; d2 = td;
                    const int tj = j1; j1 = j2; j2 = tj;
                    if (k == 0 && qv) ++swaps;
                }
            }
            if (k == 0 && qv) {
                const int64_t row = t.row + c;
                bool pass = false;
                if (j2 >= 0) pass = ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, ml.ratio_lo, ml.ratio_hi, rechecks);
                ml.out.best_j[row] = pass ? j1 : -1;
                if (ml.out.d1sq) ml.out.d1sq[row] = d1;
                if (ml.out.d2sq) ml.out.d2sq[row] = d2;
                matches += pass ? 1u : 0u;
            }
            return true;
        };
        // ping-pong between two register sets: inputs prefetched one sub-tile ahead are
        // never copied (a copy would wait for the load)
        SubTile tA{}, tB{};
        In vA{}, vB{};
        int iA = 0, iB = 0;
        bool hA = next(tA, iA), hB = false;
        if (hA) vA = fetch(tA);
        bool ok = true;
        while (hA) {
            hB = next(tB, iB);
            if (hB) vB = fetch(tB);
            if (!process(tA, vA, iA)) { ok = false; break; }
            if (!hB) break;
            hA = next(tA, iA);
            if (hA) vA = fetch(tA);
            if (!process(tB, vB, iB)) { ok = false; break; }
        }
        if (!ok) give_up();
        if (ml.out.stats) {
            if (rechecks) atomicAdd(&s_stats[0], rechecks);
            if (matches) atomicAdd(&s_stats[1], matches);
            if (swaps) atomicAdd(&s_stats[2], swaps);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (ml.out.stats && tid == 0) {
        if (s_stats[0]) atomicAdd(&ml.out.stats[0], s_stats[0]);
        if (s_stats[1]) atomicAdd(&ml.out.stats[1], s_stats[1]);
        if (s_stats[2]) atomicAdd(&ml.out.stats[2], s_stats[2]);
    }
    if (warp == C::MMA_WARP) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 256);
    }
}

// One row per 8 threads (16 descriptor bytes each): BF16 or scaled-E4M3 copy.
template <bool FP8>
__global__ void __launch_bounds__(256) k_xcopy(HashLaunch h) {
    const int64_t rows_per_block = 256 / 8;
    for (int tile = blockIdx.x; tile < h.n_tiles; tile += gridDim.x) {
        int lo = 0, hi = h.n_batch;  // image of this 64-row tile
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (h.tile_pref[mid] <= tile) lo = mid; else hi = mid;
        }
        const DevImage e = h.imgs[h.batch[lo]];
        const int row0 = (tile - h.tile_pref[lo]) * kHashTile;
        for (int rr = threadIdx.x >> 3; rr < kHashTile; rr += (int)rows_per_block) {
            const int row = row0 + rr, seg = threadIdx.x & 7;
            const bool ok = row < e.n;   // uniform over the 8 lanes of a row
            uint4 v = make_uint4(0, 0, 0, 0);
            if (ok) v = __ldg(reinterpret_cast<const uint4*>(e.desc + (size_t)row * kDim) + seg);
            if (!FP8) {
                if (ok) {
                    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                    uint32_t o[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint32_t b0 = (w[q >> 1] >> (16 * (q & 1))) & 0xFFu;
                        const uint32_t b1 = (w[q >> 1] >> (16 * (q & 1) + 8)) & 0xFFu;
                        // an integer 0..255 is exact in BF16: the upper half of its FP32 value
                        o[q] = (__float_as_uint((float)b0) >> 16) | (__float_as_uint((float)b1) & 0xFFFF0000u);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(static_cast<unsigned char*>(e.xq) + (size_t)row * 256 + seg * 32);
                    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
                    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
                }
            } else {
                uint32_t mx = __vmaxu4(__vmaxu4(v.x, v.y), __vmaxu4(v.z, v.w));
                mx = __vmaxu4(mx, mx >> 16);
                mx = __vmaxu4(mx, mx >> 8);
                mx &= 0xFFu;
                mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 1));
                mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 2));
                mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 4));
                if (ok) {
                    const float scale = mx ? (float)mx / 448.f : 1.f;
                    const float inv = 1.f / scale;
                    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                    uint32_t o[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float f0 = (float)(w[q] & 0xFFu) * inv, f1 = (float)((w[q] >> 8) & 0xFFu) * inv;
                        const float f2 = (float)((w[q] >> 16) & 0xFFu) * inv, f3 = (float)(w[q] >> 24) * inv;
                        const uint32_t lo2 = __nv_cvt_float2_to_fp8x2(make_float2(f0, f1), __NV_SATFINITE, __NV_E4M3);
                        const uint32_t hi2 = __nv_cvt_float2_to_fp8x2(make_float2(f2, f3), __NV_SATFINITE, __NV_E4M3);
                        o[q] = lo2 | (hi2 << 16);
                    }
                    *reinterpret_cast<uint4*>(static_cast<unsigned char*>(e.xq) + (size_t)row * 128 + seg * 16) =
                        make_uint4(o[0], o[1], o[2], o[3]);
                    if (seg == 0) e.xscale[row] = scale;
                }
            }
        }
    }
}

template <int K, bool FP8>
cudaError_t launch_rr(const MatchLaunch& m, int sms, cudaStream_t s) {
    using C = RR<K, FP8>;
    cudaError_t e = cudaFuncSetAttribute(k_rerank_tc<K, FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const int n_sub = m.n_items * (m.S / C::QS);
    const int slots = C::CTAS * sms;
    const int grid = n_sub < slots ? (n_sub ? n_sub : 1) : slots;
    k_rerank_tc<K, FP8><<<grid, C::THREADS, C::SMEM, s>>>(m);
    return cudaGetLastError();
}

template <bool FP8>
cudaError_t launch_rr_k(const MatchLaunch& m, int sms, cudaStream_t s) {
    switch (m.K) {
        case 2: return launch_rr<2, FP8>(m, sms, s);
        case 4: return launch_rr<4, FP8>(m, sms, s);
        case 8: return launch_rr<8, FP8>(m, sms, s);
        case 16: return launch_rr<16, FP8>(m, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_xcopy(const HashLaunch& h, cudaStream_t s) {
    if (h.n_tiles == 0) return cudaSuccess;
    const int grid = h.n_tiles < 4096 ? h.n_tiles : 4096;
    if (h.rerank == CM_RERANK_FP8) k_xcopy<true><<<grid, 256, 0, s>>>(h);
    else k_xcopy<false><<<grid, 256, 0, s>>>(h);
    return cudaGetLastError();
}

cudaError_t launch_rerank_tc(const MatchLaunch& m, int sm_count, cudaStream_t s) {
    if (m.n_items == 0) return cudaSuccess;
    return m.rerank == CM_RERANK_FP8 ? launch_rr_k<true>(m, sm_count, s) : launch_rr_k<false>(m, sm_count, s);
}

}  // namespace cm
