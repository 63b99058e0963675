// kern_step.cu -- the integer/gather stages of one time step (sm_103a):
//   a1 truncation Q (threshold keep bits and their scan; the kept set is then
//      sorted and placed by kern_sort.cu),
//   a2/a3 one BFS level of H_eff: expansion of the frontier through H's moves,
//         hash de-duplication with first-occurrence winners, compaction,
//   a4 rescue of re-admitted amplitudes from the previous step's table,
//   a5 the restricted Hamiltonian P_m H P_m, row-pitched,
//   a7 observables.
// Paper: Sec. 3.3 (neighbour sets, Eqs. def_neighbor/def_neighbor_k/H_eff;
// truncation and post-adaptation detruncation; generating the effective
// Hamiltonian) and Sec. 3.4 (the step map).
#include <type_traits>

#include "runtime.h"
#include "paces.h"

namespace paces {

// Contiguous chunk of [0, n) for block b of G, aligned to the block size so
// that 32-row bitmask words never straddle chunks.


// ---------------------------------------------------------------- insert rows
template <int W>
__global__ void k_insert_rows(const uint64_t* __restrict__ keys, uint32_t n, uint64_t* table, uint64_t slots,
                              Counters* ctr)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, i);
        if (!table_insert_unique<W>(table, slots, k, i)) set_err(ctr, kErrProbe, -1, 0);
    }
}

// ---------------------------------------------------------------- a1 truncation
// keep_i = re^2 + im^2 >= theta^2.  FP64 storage: evaluated in FP64 with every
// product and sum rounded separately (no FMA contraction), as the oracle does.
// Double-word storage: |c|^2 in double-word arithmetic (relative error below
// 2^-46) compared with theta^2 rounded to a double-word.
//
// FP64 storage: the FP64 pipe of this part retires about two operations per SM
// and clock, so the three FP64 operations of the test would bound the pass.
// The decision is first taken from the leading 20 bits of each component
// (mag_scaled_f32, integer operations, scaled by 2^(32 - L) so that theta^2
// lands near 1 in FP32): a = |x| 2^(32-L), b = |y| 2^(32-L), each at most
// 2^-20 below the exact magnitude, so a^2 + b^2 (FP32, three roundings of
// 2^-24) is within 2^-18 of |c|^2 2^(64-2L), and the FP64 test's own rounding is
// 2^-52.  Outside a band of 2^-14 around t = theta^2 2^(64-2L) the decision is
// therefore the FP64 test's; inside it, for infinite or NaN components and
// for theta^2 outside [2^-400, 2^100] (where t would leave the FP32 range),
// the FP64 test runs.  The kept set is the same bit for bit.
struct KeepTest {
    double th2;
    int L;          // scale exponent: t = theta^2 2^(64 - 2L) in [1/4, 1)
    bool filter;    // false: FP64 test only
    float t_lo, t_hi;
};

__device__ __forceinline__ KeepTest keep_test(double th2)
{
    KeepTest k;
    k.th2 = th2;
    k.filter = th2 >= 0x1p-400 && th2 <= 0x1p100;
    k.L = 32;
    k.t_lo = k.t_hi = 0.f;
    if (k.filter) {
        const int E = ilogb(th2);               // th2 in [2^E, 2^(E+1))
        k.L = 32 + ((E + 2) >> 1);              // 2 (L - 32) = E + 1 or E + 2 (floor division)
        const float t = (float)ldexp(th2, 64 - 2 * k.L);
        k.t_lo = t * (1.0f - 0x1p-14f);
        k.t_hi = t * (1.0f + 0x1p-14f);
    }
    return k;
}

__device__ __forceinline__ bool keep_row(const double2* c, uint64_t i, int fmt, const KeepTest& kt, dwf th)
{
    if (fmt == 1) {
        double2 v = c[i];
        const int ex = (__double2hiint(v.x) >> 20) & 0x7FF, ey = (__double2hiint(v.y) >> 20) & 0x7FF;
        if (kt.filter && ex != 0x7FF && ey != 0x7FF) {
            const float a = mag_scaled_f32(v.x, kt.L), b = mag_scaled_f32(v.y, kt.L);
            const float w = __fmaf_rn(a, a, __fmul_rn(b, b));
            if (w < kt.t_lo) return false;
            if (w > kt.t_hi) return true;
        }
        return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)) >= kt.th2;
    }
    dwf w = dw_norm2(reinterpret_cast<const float4*>(c)[i]);
    return w.hi > th.hi || (w.hi == th.hi && w.lo >= th.lo);
}

__global__ void __launch_bounds__(kBlock) k_trunc_count(const double2* __restrict__ c, Counters* ctr, double th2,
                                                        dwf th, int fmt, uint32_t* __restrict__ keepw,
                                                        uint32_t* __restrict__ blk_cnt)
{
    if (ctr->err) return;
    uint32_t q = ctr->q, lo, hi;
    chunk_of(q, gridDim.x, blockIdx.x, lo, hi);
    const KeepTest kt = keep_test(th2);
    uint32_t cnt = 0;
    for (uint32_t base = lo; base < hi; base += kBlock) {
        uint32_t i = base + threadIdx.x;
        bool keep = (i < hi) && keep_row(c, i, fmt, kt, th);
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        uint32_t w0 = base + (threadIdx.x & ~31u);
        if ((threadIdx.x & 31) == 0 && w0 < hi) keepw[w0 >> 5] = bal;
        cnt += keep ? 1u : 0u;
    }
    uint32_t tot;
    block_excl_scan<kBlock>(cnt, &tot);
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = tot;
}

enum ScanMode { kScanTrunc = 0, kScanLevel = 1 };

// Exclusive scan of the chunk counts; publishes the new row count.
__global__ void __launch_bounds__(1024) k_scan(const uint32_t* __restrict__ blk_cnt, uint32_t* __restrict__ blk_off,
                                               int G, Counters* ctr, int mode, int f, uint32_t cap_rows, int step)
{
    if (ctr->err) return;
    uint32_t v = threadIdx.x < (unsigned)G ? blk_cnt[threadIdx.x] : 0u;
    uint32_t tot;
    uint32_t ex = block_excl_scan<1024>(v, &tot);
    if (threadIdx.x < (unsigned)G) blk_off[threadIdx.x] = ex;
    if (threadIdx.x == 0) {
        if (mode == kScanTrunc) {
            ctr->q_in = ctr->q;
            ctr->kept = tot;
            ctr->q = tot;
            ctr->level_off[0] = 0;
            ctr->level_off[1] = tot;
            ctr->nlevels = 1;
        } else {
            uint64_t hi = ctr->level_off[f + 1];
            uint64_t nq = hi + tot;
            if (nq > cap_rows || f + 2 > kMaxLevels + 1) {
                set_err(ctr, kErrRows, step, (int)f);
            } else {
                ctr->level_off[f + 2] = (uint32_t)nq;
                ctr->q = (uint32_t)nq;
                ctr->nlevels = f + 2;
            }
        }
    }
}

// ---------------------------------------------------------------- a2/a3 one level
// Candidate c = (parent p - lo) * D + move: the parents of a level are the
// frontier rows [lo, hi); every candidate is inserted independently.  Each
// thread takes kCPT candidates at once and issues their parent loads, moves
// and home-slot loads before resolving any of them, so that a warp keeps
// 32 kCPT probe sequences in flight instead of waiting on one dependent
// chain (parent, move, hash, DRAM probe, atomic) at a time.
//
// The home slot of a key and its contents, loaded ahead of the probe loop.
struct Probe {
    uint64_t pos, fp, tag, kw;
};

template <int W>
__device__ __forceinline__ void probe_start(const uint64_t* table, uint64_t slots, const Key<W>& key, Probe& pr)
{
    const uint64_t h = key_hash<W>(key);
    pr.fp = fingerprint<W>(h);
    pr.pos = slot_home(h, slots);
    const uint64_t* sl = table + pr.pos * Slot<W>::kWords;
    if constexpr (W == 1) {
        ulonglong2 s2 = __ldcg(reinterpret_cast<const ulonglong2*>(sl));
        pr.tag = s2.x;
        pr.kw = s2.y;
    } else {
        pr.tag = __ldcg(sl);
        pr.kw = kEmpty;
    }
}

//
// Insert a candidate.  Returns the slot that holds its key afterwards: a slot
// it claimed, a candidate entry with the same key it joined (the lowest
// candidate index wins, through atomicMin on the tag), or the slot of an
// existing row.  kNone only on failure.  The slot is recorded per (parent row,
// move), so the P H P build later reads the column of every move of a
// non-final level from it without probing.
template <int W>
__device__ __forceinline__ uint32_t insert_candidate(const DevModel* __restrict__ M, uint64_t* table, uint64_t slots,
                                                     const Key<W>& key, uint32_t c, const uint64_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ meta, uint32_t lo, Counters* ctr,
                                                     int step, const Probe& pr, bool& resolved)
{
    const uint64_t fp = pr.fp;
    uint64_t mine = (fp << 32) | (uint64_t)(kCand | c);
    uint64_t pos = pr.pos;
    resolved = false;
    for (uint32_t probe = 0; probe < kMaxProbe; ++probe) {
        uint64_t* sl = table + pos * Slot<W>::kWords;
        uint64_t tag, kw = kEmpty;
        if constexpr (W == 1) {
            // a one-word slot is claimed with its key in one 16-byte atomic, so
            // a later candidate of the same key compares the key in the slot
            ulonglong2 s2 = probe == 0 ? make_ulonglong2(pr.tag, pr.kw)
                                       : __ldcg(reinterpret_cast<const ulonglong2*>(sl));
            tag = s2.x;
            kw = s2.y;
            if (tag == kEmpty) {
                uint64_t olo, ohi;
                cas128(sl, kEmpty, kEmpty, mine, key.w[0], olo, ohi);
                if (olo == kEmpty) return (uint32_t)pos;
                tag = olo;
                kw = ohi;
            }
        } else {
            tag = probe == 0 ? pr.tag : __ldcg(sl);
            if (tag == kEmpty) {
                unsigned long long old = atomicCAS((unsigned long long*)sl, kEmpty, mine);
                if (old == kEmpty) return (uint32_t)pos;
                tag = old;
            }
        }
        if ((tag >> 32) == fp) {
            uint32_t v = (uint32_t)tag;
            if (W == 1 && (v & kCand) && kw != kEmpty) {
                if (kw == key.w[0]) {
                    atomicMin((unsigned long long*)sl, (unsigned long long)mine);
                    return (uint32_t)pos;
                }
            } else if (v & kCand) {
                // another candidate holds the slot: regenerate its key from its parent
                uint32_t c2 = v & ~kCand;
                uint32_t p2 = (uint32_t)udiv(c2, M->div_D);
                int mv2 = (int)(c2 - p2 * (uint32_t)M->D);
                Key<W> pk = load_key<W>(keys, lo + p2);
                uint32_t pm = meta[lo + p2];
                Key<W> k2;
                int cid2;
                if (apply_move<W>(M, pk, meta_s(pm), meta_ns(pm), mv2, k2, cid2) && key_eq<W>(k2, key)) {
                    atomicMin((unsigned long long*)sl, (unsigned long long)mine);
                    return (uint32_t)pos;
                }
            } else {
                bool eq = true;
#pragma unroll
                for (int i = 0; i < W; ++i) eq &= (__ldcg(sl + 1 + i) == key.w[i]);
                if (eq) {
                    resolved = true;          // an existing row: return it
                    return v;
                }
            }
        }
        pos = slot_next(pos, slots);
    }
    set_err(ctr, kErrProbe, step, 2);
    return kNone;
}

// Lookup continuing from a loaded home slot in a table that does not change
// while the kernel runs (the previous step's): row of key or -1.
template <int W>
__device__ __forceinline__ int64_t lookup_from(const uint64_t* __restrict__ table, uint64_t slots, const Key<W>& key,
                                               const Probe& pr)
{
    uint64_t pos = pr.pos;
    for (uint32_t probe = 0; probe < kMaxProbe; ++probe) {
        const uint64_t* sl = table + pos * Slot<W>::kWords;
        uint64_t tag, kw;
        if constexpr (W == 1) {
            ulonglong2 s2 = probe == 0 ? make_ulonglong2(pr.tag, pr.kw) : __ldg(reinterpret_cast<const ulonglong2*>(sl));
            tag = s2.x;
            kw = s2.y;
        } else {
            tag = probe == 0 ? pr.tag : __ldg(sl);
            kw = kEmpty;
        }
        if (tag == kEmpty) return -1;
        if ((tag >> 32) == pr.fp) {
            bool eq;
            if constexpr (W == 1) {
                eq = kw == key.w[0];
            } else {
                eq = true;
#pragma unroll
                for (int i = 0; i < W; ++i) eq &= (__ldg(sl + 1 + i) == key.w[i]);
            }
            if (eq) return (int64_t)(uint32_t)tag;
        }
        pos = slot_next(pos, slots);
    }
    return -1;
}

// Candidate c of the level whose frontier starts at row lo: parent row and move.
__device__ __forceinline__ void cand_parent(const DevModel* __restrict__ M, uint32_t c, uint32_t lo, uint32_t& p,
                                            int& mv)
{
    uint32_t pl = (uint32_t)udiv(c, M->div_D);
    mv = (int)(c - pl * (uint32_t)M->D);
    p = lo + pl;
}

// One-word keys: the kCPT candidates of a thread are inserted in lockstep.
// Every round first claims, with one 16-byte compare-and-swap each, all the
// empty slots its candidates stand on, then compares every occupied slot's key
// with its candidate's (a one-word slot holds the key next to the tag): the
// same key as another candidate's joins it (atomicMin on the tag, the lowest
// candidate index wins), the same key as an existing row resolves to that row,
// and a different key moves to the next slot, whose load is issued with the
// others of the round.  All lanes run the same instructions (predicated), so a
// warp keeps its 32 kCPT claims or probe loads in flight together instead of
// resolving one candidate's chain (load, compare, claim) after another's.
constexpr int kCPT1 = 4;                    // one-word keys: candidates per thread
__device__ __forceinline__ void insert_lockstep(uint64_t* table, uint64_t slots, const Key<1> (&child)[kCPT1],
                                                uint32_t c0, uint32_t stride, const bool (&ok)[kCPT1],
                                                const Probe (&pb)[kCPT1], Counters* ctr, int step,
                                                const uint32_t (&pp)[kCPT1], const int (&mvv)[kCPT1], int D,
                                                uint32_t nc, uint32_t* __restrict__ cand_slot)
{
    constexpr int kCPT = kCPT1;
    uint32_t pos[kCPT], res[kCPT];
    uint64_t tag[kCPT], kw[kCPT];
    unsigned act = 0;                               // bit k: candidate k unresolved
#pragma unroll
    for (int k = 0; k < kCPT; ++k) {
        pos[k] = (uint32_t)pb[k].pos;               // slots < 2^32
        tag[k] = pb[k].tag;
        kw[k] = pb[k].kw;
        res[k] = kNone;
        act |= ok[k] ? (1u << k) : 0u;
    }
    for (uint32_t round = 0; round <= kMaxProbe; ++round) {
        if (!__any_sync(0xffffffffu, act != 0)) break;
        unsigned tried = 0;
#pragma unroll
        for (int k = 0; k < kCPT; ++k)              // claims of empty slots, all in flight
            if (((act >> k) & 1u) && tag[k] == kEmpty) {
                const uint64_t mine = (pb[k].fp << 32) | (uint64_t)(kCand | (c0 + (uint32_t)k * stride));
                cas128(table + (uint64_t)pos[k] * 2, kEmpty, kEmpty, mine, child[k].w[0], tag[k], kw[k]);
                tried |= 1u << k;
            }
        unsigned adv = 0;
#pragma unroll
        for (int k = 0; k < kCPT; ++k) {
            if (!((act >> k) & 1u)) continue;
            if (((tried >> k) & 1u) && tag[k] == kEmpty) {   // claimed (the old tag was empty)
                res[k] = pos[k];
                act &= ~(1u << k);
                continue;
            }
            // occupied, or lost the race: tag and kw hold the slot's entry
            if (kw[k] == child[k].w[0]) {
                const uint32_t v = (uint32_t)tag[k];
                if (v & kCand) {                    // another candidate of this key
                    const uint64_t mine = (pb[k].fp << 32) | (uint64_t)(kCand | (c0 + (uint32_t)k * stride));
                    atomicMin((unsigned long long*)(table + (uint64_t)pos[k] * 2), (unsigned long long)mine);
                    res[k] = pos[k];
                } else {
                    res[k] = kCand | v;             // an existing row
                }
                act &= ~(1u << k);
            } else {
                pos[k] = (uint32_t)slot_next(pos[k], slots);
                adv |= 1u << k;
            }
        }
#pragma unroll
        for (int k = 0; k < kCPT; ++k)              // next slots, all in flight
            if ((adv >> k) & 1u) {
                const ulonglong2 s2 = __ldcg(reinterpret_cast<const ulonglong2*>(table + (uint64_t)pos[k] * 2));
                tag[k] = s2.x;
                kw[k] = s2.y;
            }
    }
#pragma unroll
    for (int k = 0; k < kCPT; ++k) {
        const uint32_t c = c0 + (uint32_t)k * stride;
        if (c >= nc) continue;
        if ((act >> k) & 1u) set_err(ctr, kErrProbe, step, 2);
        cand_slot[(uint64_t)pp[k] * D + mvv[k]] = res[k];
    }
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_level_insert(const DevModel* __restrict__ M, Counters* ctr, int f,
                                                         const uint64_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ meta, uint64_t* table,
                                                         uint64_t slots, uint32_t* __restrict__ cand_slot,
                                                         uint64_t cand_cap, int step)
{
    if (ctr->err) return;
    uint32_t lo = ctr->level_off[f], hi = ctr->level_off[f + 1];
    const int D = M->D;
    uint64_t ncand = (uint64_t)(hi - lo) * (uint64_t)D;
    if (ncand >= (uint64_t)kCand || (uint64_t)hi * D > cand_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctr, kErrCand, step, f);
        return;
    }
    constexpr int kCPT = W == 1 ? kCPT1 : 2;
    const uint32_t nc = (uint32_t)ncand, stride = gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of rounds (the lockstep
    // insertion votes over the whole warp); lanes past nc have no candidates
    for (uint32_t cw = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); cw < nc; cw += stride * kCPT) {
        const uint32_t c0 = cw + (threadIdx.x & 31u);
        Key<W> child[kCPT];
        Probe pb[kCPT] = {};
        uint32_t pp[kCPT];
        int mvv[kCPT];
        bool ok[kCPT];
#pragma unroll
        for (int k = 0; k < kCPT; ++k) {        // parents and moves
            const uint32_t c = c0 + (uint32_t)k * stride;
            ok[k] = false;
            pp[k] = 0;
            mvv[k] = 0;
            if (c < nc) {
                cand_parent(M, c, lo, pp[k], mvv[k]);
                const Key<W> pk = load_key<W>(keys, pp[k]);
                const uint32_t pm = meta[pp[k]];
                int cid;
                ok[k] = apply_move<W>(M, pk, meta_s(pm), meta_ns(pm), mvv[k], child[k], cid);
            }
        }
#pragma unroll
        for (int k = 0; k < kCPT; ++k)          // every home slot in flight at once
            if (ok[k]) probe_start<W>(table, slots, child[k], pb[k]);
        if constexpr (W == 1) {
            insert_lockstep(table, slots, child, c0, stride, ok, pb, ctr, step, pp, mvv, D, nc, cand_slot);
        } else {
#pragma unroll
            for (int k = 0; k < kCPT; ++k) {
                const uint32_t c = c0 + (uint32_t)k * stride;
                if (c >= nc) continue;
                uint32_t r = kNone;
                bool res = false;
                if (ok[k]) r = insert_candidate<W>(M, table, slots, child[k], c, keys, meta, lo, ctr, step, pb[k], res);
                cand_slot[(uint64_t)pp[k] * D + mvv[k]] = res ? (kCand | r) : r;
            }
        }
    }
}

// Winner bits, one per candidate (32 per word, chunks aligned to 256).  A
// block takes kR rounds of kBlock candidates at once: the candidate-slot reads
// of all rounds, then the tag reads of all rounds, are issued before any
// winner is decided, so each thread keeps kR dependent pairs in flight.
template <int W>
__global__ void __launch_bounds__(kBlock) k_level_flags(const DevModel* __restrict__ M, Counters* ctr, int f,
                                                        const uint64_t* __restrict__ table,
                                                        const uint32_t* __restrict__ cand_slot,
                                                        uint32_t* __restrict__ wmask, uint32_t* __restrict__ blk_cnt)
{
    constexpr int kR = 4;
    if (ctr->err) return;
    uint32_t lo0 = ctr->level_off[f], NC = (ctr->level_off[f + 1] - lo0) * (uint32_t)M->D, lo, hi;
    chunk_of(NC, gridDim.x, blockIdx.x, lo, hi);
    const int D = M->D;
    uint32_t cnt = 0;
    for (uint32_t base = lo; base < hi; base += kBlock * kR) {
        uint32_t sl[kR], tg[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const uint32_t c = base + (uint32_t)r * kBlock + threadIdx.x;
            sl[r] = kNone;
            if (c < hi) {
                uint32_t p;
                int mv;
                cand_parent(M, c, lo0, p, mv);
                sl[r] = cand_slot[(uint64_t)p * D + mv];
            }
        }
        // a candidate that met an existing row (kCand | row), or none, is no
        // winner: no tag read
#pragma unroll
        for (int r = 0; r < kR; ++r)
            tg[r] = (sl[r] & kCand) ? 0u : (uint32_t)table[(uint64_t)sl[r] * Slot<W>::kWords];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const uint32_t c = base + (uint32_t)r * kBlock + threadIdx.x;
            const bool win = c < hi && !(sl[r] & kCand) && tg[r] == (kCand | c);
            const unsigned bal = __ballot_sync(0xffffffffu, win);
            const uint32_t w0 = base + (uint32_t)r * kBlock + (threadIdx.x & ~31u);
            if ((threadIdx.x & 31) == 0 && w0 < hi) wmask[w0 >> 5] = bal;
            cnt += win ? 1u : 0u;
        }
    }
    uint32_t tot;
    block_excl_scan<kBlock>(cnt, &tot);
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = tot;
}

// New rows in candidate order: key, descriptor, table slot (key words + row).
// The winners of each round of kBlock candidates (a minority: most candidates
// meet a row or another candidate of their key) are queued in shared memory in
// candidate order and written out once kBlock of them are pending, so that
// every lane of a warp builds a row instead of the few that won their round.
template <int W>
__global__ void __launch_bounds__(kBlock) k_level_scatter(const DevModel* __restrict__ M, Counters* ctr, int f,
                                                          uint64_t* keys, uint32_t* meta, uint64_t* table,
                                                          const uint32_t* __restrict__ cand_slot,
                                                          const uint32_t* __restrict__ wmask,
                                                          const uint32_t* __restrict__ blk_off)
{
    constexpr int kCPT = 4;                     // consecutive candidates per thread and round
    constexpr uint32_t kRound = kBlock * kCPT;
    __shared__ uint32_t qc[kRound + kBlock];
    if (ctr->err) return;
    uint32_t lo0 = ctr->level_off[f], base_row = ctr->level_off[f + 1];
    const int D = M->D;
    uint32_t NC = (base_row - lo0) * (uint32_t)D, lo, hi;
    chunk_of(NC, gridDim.x, blockIdx.x, lo, hi);
    uint32_t run = blk_off[blockIdx.x];
    uint32_t pending = 0;
    // at most kRound + kBlock - 1 rows are pending: every thread loads the
    // parents (key, descriptor, candidate slot) of kPT of its rows, then builds
    // them (one-word keys: all its rows at once)
    constexpr int kPT = W == 1 ? (kRound + kBlock) / kBlock : 2;
    auto write_rows = [&](uint32_t n) {
        for (uint32_t i0 = threadIdx.x; i0 < n; i0 += kPT * kBlock) {
            Key<W> pk[kPT];
            uint32_t pm[kPT], sl[kPT];
            int mvv[kPT];
#pragma unroll
            for (int u = 0; u < kPT; ++u) {
                const uint32_t i = i0 + (uint32_t)u * kBlock;
                if (i >= n) continue;
                uint32_t p;
                int mv;
                cand_parent(M, qc[i], lo0, p, mv);
                mvv[u] = mv;
                pk[u] = load_key<W>(keys, p);
                pm[u] = meta[p];
                sl[u] = cand_slot[(uint64_t)p * D + mv];
            }
#pragma unroll
            for (int u = 0; u < kPT; ++u) {
                const uint32_t i = i0 + (uint32_t)u * kBlock;
                if (i >= n) continue;
                const Key<W> k = pk[u];
                Key<W> child;
                int cid;
                apply_move<W>(M, k, meta_s(pm[u]), meta_ns(pm[u]), mvv[u], child, cid);
                const uint32_t row = base_row + run + i;
                store_key<W>(keys, row, child);
                meta[row] = child_meta<W>(M, k, pm[u], mvv[u]);
                uint64_t* slp = table + (uint64_t)sl[u] * Slot<W>::kWords;
                // the tag is rebuilt from the key's hash: a store, no read of the slot
                const uint64_t tag = ((uint64_t)fingerprint<W>(key_hash<W>(child)) << 32) | (uint64_t)row;
                if constexpr (W == 1) {
                    *reinterpret_cast<ulonglong2*>(slp) = make_ulonglong2(tag, child.w[0]);
                } else {
#pragma unroll
                    for (int w = 0; w < W; ++w) slp[1 + w] = child.w[w];
                    slp[0] = tag;
                }
            }
        }
    };
    // chunks are multiples of kBlock candidates (chunk_of), so a thread's four
    // consecutive candidates share one 32-bit mask word
    for (uint32_t base = lo; base < hi; base += kRound) {
        const uint32_t c = base + kCPT * threadIdx.x;
        unsigned bits = 0;
        if (c < hi) {
            bits = (wmask[c >> 5] >> (c & 31u)) & 0xFu;
            if (hi - c < (uint32_t)kCPT) bits &= (1u << (hi - c)) - 1u;
        }
        uint32_t tot;
        const uint32_t r = block_excl_scan<kBlock>((uint32_t)__popc(bits), &tot);
        uint32_t o = pending + r;
#pragma unroll
        for (int k = 0; k < kCPT; ++k)
            if ((bits >> k) & 1u) qc[o++] = c + (uint32_t)k;
        pending += tot;
        if (pending >= kBlock) {
            __syncthreads();
            write_rows(pending);
            run += pending;
            pending = 0;
            __syncthreads();
        }
    }
    if (pending) {
        __syncthreads();
        write_rows(pending);
    }
}

// Rescue (post-adaptation detruncation, Sec. 3.3) of the rows a level added:
// each takes its amplitude from the previous step's table when its key was a
// row there, else 0 (also 0 with no previous table).  Dense over the new rows;
// each thread takes kRPT rows and issues their home-slot loads, then their
// amplitude gathers, together.
template <int W>
__global__ void __launch_bounds__(kBlock) k_level_rescue(const Counters* __restrict__ ctr, int f,
                                                         const uint64_t* __restrict__ keys,
                                                         const uint64_t* __restrict__ old_table, uint64_t old_slots,
                                                         const double2* __restrict__ c_old, double2* __restrict__ c_new,
                                                         uint32_t* __restrict__ from)
{
    if (ctr->err) return;
    constexpr int kRPT = W == 1 ? 4 : 2;
    const uint32_t lo = ctr->level_off[f + 1], hi = ctr->level_off[f + 2];
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r0 = lo + blockIdx.x * blockDim.x + threadIdx.x; r0 < hi; r0 += stride * kRPT) {
        Key<W> key[kRPT];
        Probe pb[kRPT];
        int64_t orow[kRPT];
#pragma unroll
        for (int k = 0; k < kRPT; ++k) {
            const uint32_t row = r0 + (uint32_t)k * stride;
            orow[k] = -1;
            if (row < hi) {
                key[k] = load_key<W>(keys, row);
                if (old_table) probe_start<W>(old_table, old_slots, key[k], pb[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kRPT; ++k) {
            const uint32_t row = r0 + (uint32_t)k * stride;
            if (row < hi && old_table) orow[k] = lookup_from<W>(old_table, old_slots, key[k], pb[k]);
        }
        double2 a[kRPT];
#pragma unroll
        for (int k = 0; k < kRPT; ++k) a[k] = orow[k] >= 0 ? c_old[orow[k]] : make_double2(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < kRPT; ++k) {
            const uint32_t row = r0 + (uint32_t)k * stride;
            if (row >= hi) continue;
            c_new[row] = a[k];
            if (from) from[row] = orow[k] >= 0 ? (uint32_t)orow[k] : kNone;
        }
    }
}

// ---------------------------------------------------------------- a5 P H P
// Row i holds the off-diagonal entries of P_m H P_m in move order (hops to
// t ascending, a_s^dag, a_s), columns = rows of the images that lie in H_eff,
// and the diagonal eps_s + sum_j omega_j n_j.  Rows of every level except the
// last were expanded: each of their valid moves is in H_eff and its slot was
// recorded, so the column is one read of that slot's tag; rows of the last
// level probe the table.
struct DiagAcc {
    double d;      // FP64 diagonal: eps_s + omega N_ph (one rounding) when every
                   // omega_j is equal, else summed in site order
    dwf dd;        // double-word diagonal
};

template <int W>
__device__ __forceinline__ DiagAcc row_diag(const DevModel* __restrict__ M, const Key<W>& k, int s, int nph)
{
    double e64 = M->eps[s];
    dwf edw = M->eps_dw[s];
    if (M->batch > 1) {                         // site energies of this key's realisation
        int rz = key_real<W>(k, M);
        e64 = M->eps_b64[rz * M->N + s];
        edw = M->eps_bdw[rz * M->N + s];
    }
    if (M->uniform_omega) {                   // eps_s + omega N_ph, no digits needed
        DiagAcc r{0.0, {0.f, 0.f}};
        if (M->fmt == 1) r.d = fma(M->omega[0], (double)nph, e64);
        else r.dd = dw_add(edw, dw_mul_f(M->omega_dw[0], (float)nph));
        return r;
    }
    uint64_t q0 = udiv(k.w[0], M->div_exc);
    DiagAcc r{e64, edw};
    const bool f64 = M->fmt == 1;
    nph = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t x = (w == 0) ? q0 : k.w[w];
        for (int j = M->word_first[w]; j < M->word_first[w + 1]; ++j) {
            uint64_t xq = udiv(x, M->div_radix[j]);
            int nj = (int)(x - xq * M->div_radix[j].d);
            x = xq;
            if (f64) r.d = __dadd_rn(r.d, __dmul_rn(M->omega[j], (double)nj));
            else if (!M->uniform_omega && nj) r.dd = dw_add(r.dd, dw_mul_f(M->omega_dw[j], (float)nj));
            nph += nj;
        }
    }
    if (!f64 && M->uniform_omega) r.dd = dw_add(r.dd, dw_mul_f(M->omega_dw[0], (float)nph));
    return r;
}

// Row bound used to choose the number of Taylor series of a step (a6):
// up20(|eps_s|) + sum_j up20(|omega_j|) n_j + up20 of every off-diagonal
// element of H in the row (hops and ladder moves, in H_eff or not), where
// up20(x) = ceil(|x| 2^20).  The largest row sum of |H| over H_eff bounds
// ||P H P||_2; integer sums make the bound exact and free of summation order.
template <int W>
__device__ __forceinline__ unsigned long long row_hbound(const DevModel* __restrict__ M, const Key<W>& k, int s,
                                                         int ns, int nph)
{
    unsigned long long b;
    if (M->batch > 1) {
        int rz = key_real<W>(k, M);
        b = (unsigned long long)ceil(fabs(M->eps_b64[rz * M->N + s]) * 1048576.0);
    } else {
        b = M->hb_eps[s];
    }
    b += M->hb_hop[s];
    if (M->uniform_omega) {
        b += M->hb_omega[0] * (unsigned long long)nph;
    } else {
        uint64_t q0 = udiv(k.w[0], M->div_exc);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t x = (w == 0) ? q0 : k.w[w];
            for (int j = M->word_first[w]; j < M->word_first[w + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                b += M->hb_omega[j] * (x - xq * M->div_radix[j].d);
                x = xq;
            }
        }
    }
    if (M->gnz[s]) {
        if (ns < M->cap[s]) b += M->hb_coef[M->lad_cid[M->lad_off[s] + ns]];
        if (ns > 0) b += M->hb_coef[M->lad_cid[M->lad_off[s] + ns - 1]];
    }
    return b;
}

__device__ __forceinline__ void hbound_publish(Counters* ctr, unsigned long long hb)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, hb, o);
        hb = v > hb ? v : hb;
    }
    if ((threadIdx.x & 31) == 0 && hb) atomicMax(&ctr->hbound, hb);
}

__device__ __forceinline__ void store_diag(const DevModel* __restrict__ M, double* diag, uint64_t i, const DiagAcc& a)
{
    if (M->fmt == 1) diag[i] = a.d;
    else reinterpret_cast<float2*>(diag)[i] = make_float2(a.dd.hi, a.dd.lo);
}

// GS lanes per row (GS = D rounded up to a power of two, at most 32): lane mv
// resolves move mv; a ballot over the group gives each found entry its place.
template <int W, int GS>
__global__ void __launch_bounds__(kBlock) k_csr_grp(const DevModel* __restrict__ M, Counters* ctr,
                                                    const uint64_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ meta,
                                                    const uint64_t* __restrict__ table, uint64_t slots,
                                                    const uint32_t* __restrict__ cand_slot,
                                                    uint32_t* __restrict__ col, uint8_t* __restrict__ cidv,
                                                    uint8_t* __restrict__ cnt, double* __restrict__ diag)
{
    if (ctr->err) return;
    const uint32_t q = ctr->q, lim = ctr->level_off[ctr->nlevels - 1];
    const int D = M->D, P = M->P;
    constexpr uint32_t RPW = 32 / GS;
    const int lane = threadIdx.x & 31, mv = lane % GS, gbase = lane - mv;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long nnz = 0, hb = 0;
    for (uint32_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
        uint32_t row = rb + lane / GS;
        bool valid = row < q;
        Key<W> k;
#pragma unroll
        for (int i = 0; i < W; ++i) k.w[i] = 0;
        uint32_t m = 0;
        if (valid) {
            k = load_key<W>(keys, row);
            m = meta[row];
        }
        int s = meta_s(m), ns = meta_ns(m);
        bool found = false;
        uint32_t colv = 0;
        int cid = 0;
        if (valid && mv < D) {
            Key<W> child;
            if (apply_move<W>(M, k, s, ns, mv, child, cid)) {
                if (row < lim) {
                    uint32_t sl = cand_slot[(uint64_t)row * D + mv];
                    if (sl != kNone) {
                        colv = (sl & kCand) ? (sl & ~kCand) : (uint32_t)table[(uint64_t)sl * Slot<W>::kWords];
                        found = true;
                    }
                } else {
                    int64_t r = table_lookup<W>(table, slots, child);
                    if (r >= 0) {
                        colv = (uint32_t)r;
                        found = true;
                    }
                }
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, found);
        unsigned gm = (GS == 32) ? bal : ((bal >> gbase) & ((1u << GS) - 1u));
        uint64_t rbase = (uint64_t)row * P;
        if (found) {
            int pos = __popc(gm & ((1u << mv) - 1u));
            col[rbase + pos] = colv;
            cidv[rbase + pos] = (uint8_t)cid;
        }
        if (valid && mv == 0) {
            int e = __popc(gm);
            cnt[row] = (uint8_t)e;
            store_diag(M, diag, row, row_diag<W>(M, k, s, meta_nph(m)));
            unsigned long long b = row_hbound<W>(M, k, s, ns, meta_nph(m));
            hb = b > hb ? b : hb;
            nnz += e;
        }
    }
    hbound_publish(ctr, hb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    if ((threadIdx.x & 31) == 0 && nnz) atomicAdd(&ctr->nnz, nnz);
}

// One thread per row for models of at most DM (4 or 8) moves per state: every
// lane runs the same instructions for its own row.  Rows of the expanded
// levels read their D recorded slots (one vector load) and then, all together,
// the tags of the slots they name; rows of the last level look their D images
// up in lockstep rounds (every unresolved image's slot read in the same round,
// one 16-byte-aligned read per slot), so a warp keeps 32 D probes in flight.
template <int W, int DM>
__global__ void __launch_bounds__(kBlock) k_csr_row(const DevModel* __restrict__ M, Counters* ctr,
                                                    const uint64_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ meta,
                                                    const uint64_t* __restrict__ table, uint64_t slots,
                                                    const uint32_t* __restrict__ cand_slot,
                                                    uint32_t* __restrict__ col, uint8_t* __restrict__ cidv,
                                                    uint8_t* __restrict__ cnt, double* __restrict__ diag)
{
    if (ctr->err) return;
    const uint32_t q = ctr->q, lim = ctr->level_off[ctr->nlevels - 1];
    const int D = M->D, P = M->P;
    unsigned long long nnz = 0, hb = 0;
    const uint32_t nthr = gridDim.x * blockDim.x;
    for (uint32_t rb = blockIdx.x * blockDim.x; rb < q; rb += nthr) {
        const uint32_t row = rb + threadIdx.x;
        const bool valid = row < q;
        Key<W> k;
#pragma unroll
        for (int i = 0; i < W; ++i) k.w[i] = 0;
        uint32_t m = 0;
        if (valid) {
            k = load_key<W>(keys, row);
            m = meta[row];
        }
        const int s = meta_s(m), ns = meta_ns(m);
        Key<W> child[DM];
        int cid[DM];
        unsigned ok = 0, found = 0;
        uint32_t colv[DM];
#pragma unroll
        for (int mv = 0; mv < DM; ++mv) {
            cid[mv] = 0;
            colv[mv] = 0;
            if (valid && mv < D && apply_move<W>(M, k, s, ns, mv, child[mv], cid[mv])) ok |= 1u << mv;
        }
        // expanded levels: the slot (or kCand | row) every move recorded; the
        // rows of one warp may lie on both sides of lim, so both parts run as
        // predicated code and the lockstep loop below is entered by every lane
        const bool expanded = row < lim;
        {
            uint32_t sl[DM];
            const uint64_t cb = (uint64_t)row * D;
            if (DM == 4 && D == 4 && valid && expanded) {
                const uint4 v = *reinterpret_cast<const uint4*>(cand_slot + cb);
                sl[0] = v.x; sl[1] = v.y; sl[2] = v.z; sl[3] = v.w;
            } else {
#pragma unroll
                for (int mv = 0; mv < DM; ++mv)
                    sl[mv] = (expanded && ((ok >> mv) & 1u)) ? cand_slot[cb + mv] : kNone;
            }
            uint64_t tg[DM];
#pragma unroll
            for (int mv = 0; mv < DM; ++mv) {       // every slot's tag in flight at once
                tg[mv] = 0;
                if (expanded && ((ok >> mv) & 1u) && sl[mv] != kNone && !(sl[mv] & kCand))
                    tg[mv] = __ldg(table + (uint64_t)sl[mv] * Slot<W>::kWords);
            }
#pragma unroll
            for (int mv = 0; mv < DM; ++mv) {
                if (!expanded || !((ok >> mv) & 1u) || sl[mv] == kNone) continue;
                colv[mv] = (sl[mv] & kCand) ? (sl[mv] & ~kCand) : (uint32_t)tg[mv];
                found |= 1u << mv;
            }
        }
        {
            // last level: lockstep lookups of the images
            uint64_t pos[DM], fp[DM];
            unsigned act = expanded ? 0u : ok;
#pragma unroll
            for (int mv = 0; mv < DM; ++mv) {
                pos[mv] = 0;
                fp[mv] = 0;
                if ((act >> mv) & 1u) {
                    const uint64_t hsh = key_hash<W>(child[mv]);
                    fp[mv] = fingerprint<W>(hsh);
                    pos[mv] = slot_home(hsh, slots);
                }
            }
            for (uint32_t round = 0; round < kMaxProbe && __any_sync(0xffffffffu, act != 0); ++round) {
                SlotVal<W> v[DM];
#pragma unroll
                for (int mv = 0; mv < DM; ++mv)     // every unresolved image's slot in flight at once
                    if ((act >> mv) & 1u) v[mv] = read_slot<W, true>(table + pos[mv] * Slot<W>::kWords);
#pragma unroll
                for (int mv = 0; mv < DM; ++mv) {
                    if (!((act >> mv) & 1u)) continue;
                    if (v[mv].w[0] == kEmpty) {
                        act &= ~(1u << mv);          // not in H_eff
                    } else if ((v[mv].w[0] >> 32) == fp[mv] && slot_has_key<W>(v[mv], child[mv])) {
                        colv[mv] = (uint32_t)v[mv].w[0];
                        found |= 1u << mv;
                        act &= ~(1u << mv);
                    } else {
                        pos[mv] = slot_next(pos[mv], slots);
                    }
                }
            }
        }
        if (!valid) continue;
        // entries in move order, compacted
        const uint64_t rbase = (uint64_t)row * P;
        int e = 0;
        if (P == 4 && DM == 4) {
            uint32_t cc[4] = {0, 0, 0, 0}, ii = 0;
#pragma unroll
            for (int mv = 0; mv < DM; ++mv)
                if ((found >> mv) & 1u) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (t == e) cc[t] = colv[mv];
                    ii |= (uint32_t)cid[mv] << (8 * e);
                    ++e;
                }
            *reinterpret_cast<uint4*>(col + rbase) = make_uint4(cc[0], cc[1], cc[2], cc[3]);
            *reinterpret_cast<uint32_t*>(cidv + rbase) = ii;
        } else {
#pragma unroll
            for (int mv = 0; mv < DM; ++mv)
                if ((found >> mv) & 1u) {
                    col[rbase + e] = colv[mv];
                    cidv[rbase + e] = (uint8_t)cid[mv];
                    ++e;
                }
        }
        cnt[row] = (uint8_t)e;
        store_diag(M, diag, row, row_diag<W>(M, k, s, meta_nph(m)));
        const unsigned long long b = row_hbound<W>(M, k, s, ns, meta_nph(m));
        hb = b > hb ? b : hb;
        nnz += e;
    }
    hbound_publish(ctr, hb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    if ((threadIdx.x & 31) == 0 && nnz) atomicAdd(&ctr->nnz, nnz);
}

// One thread per row, for models with more than 32 moves per state.
template <int W>
__global__ void __launch_bounds__(kBlock) k_csr(const DevModel* __restrict__ M, Counters* ctr,
                                                const uint64_t* __restrict__ keys, const uint32_t* __restrict__ meta,
                                                const uint64_t* __restrict__ table,
                                                uint64_t slots, const uint32_t* __restrict__ cand_slot,
                                                uint32_t* __restrict__ col, uint8_t* __restrict__ cidv,
                                                uint8_t* __restrict__ cnt, double* __restrict__ diag)
{
    if (ctr->err) return;
    const uint32_t q = ctr->q, lim = ctr->level_off[ctr->nlevels - 1];
    const int D = M->D, P = M->P;
    unsigned long long nnz = 0, hb = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, i);
        uint32_t m = meta[i];
        int s = meta_s(m), ns = meta_ns(m);
        uint32_t e = 0;
        uint64_t rbase = (uint64_t)i * (uint64_t)P;
        for (int mv = 0; mv < D; ++mv) {
            Key<W> child;
            int cid;
            if (!apply_move<W>(M, k, s, ns, mv, child, cid)) continue;
            int64_t r = -1;
            if (i < lim) {
                uint32_t sl = cand_slot[(uint64_t)i * D + mv];
                if (sl != kNone) r = (sl & kCand) ? (sl & ~kCand) : (uint32_t)table[(uint64_t)sl * Slot<W>::kWords];
            } else {
                r = table_lookup<W>(table, slots, child);
            }
            if (r < 0) continue;
            col[rbase + e] = (uint32_t)r;
            cidv[rbase + e] = (uint8_t)cid;
            ++e;
        }
        cnt[i] = (uint8_t)e;
        store_diag(M, diag, i, row_diag<W>(M, k, s, meta_nph(m)));
        unsigned long long b = row_hbound<W>(M, k, s, ns, meta_nph(m));
        hb = b > hb ? b : hb;
        nnz += e;
    }
    hbound_publish(ctr, hb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    if ((threadIdx.x & 31) == 0 && nnz) atomicAdd(&ctr->nnz, nnz);
}

// ---------------------------------------------------------------- a7 observables
// P_s = sum over rows with site s of |c|^2, <n_j> = sum |c|^2 n_j, ||c||^2.
// Each weight w = |c|^2 is split exactly into two fixed-point integers,
// w 2^52 = hi + lo 2^-32 (hi = floor, lo = the next 32 bits), and every sum is
// an integer sum (shared-memory atomics, then per-block partials summed in
// block order): exact to 2^-84 per row, independent of scheduling, and free of
// the FP64 pipe except for the split itself.
constexpr int kObsStride = 2 * kMaxSites + 1;
constexpr size_t kObsSharedMax = 200 * 1024;

__device__ __forceinline__ void split_weight(double w, unsigned long long& hi, unsigned long long& lo)
{
    double x = w * 4503599627370496.0;          // 2^52, exact
    double f = floor(x);
    hi = (unsigned long long)f;
    lo = (unsigned long long)((x - f) * 4294967296.0);   // next 32 bits, truncated
}


// Warp sum of x as limbs of 26, 26 and 12 bits through the integer warp-reduce
// instruction (no limb sum can overflow 32 bits): three single-instruction
// reductions instead of a ten-shuffle 64-bit tree, exact modulo 2^64.
__device__ __forceinline__ unsigned long long warp_sum_limbs(unsigned long long x)
{
    const unsigned m26 = (1u << 26) - 1u;
    unsigned long long s0 = __reduce_add_sync(0xffffffffu, (unsigned)(x & m26));
    unsigned long long s1 = __reduce_add_sync(0xffffffffu, (unsigned)((x >> 26) & m26));
    unsigned long long s2 = __reduce_add_sync(0xffffffffu, (unsigned)(x >> 52));
    return s0 + (s1 << 26) + (s2 << 52);
}

// Rows are taken 32 at a time per warp.  P_s goes through atomics on the
// warp's own shared row (contention only between lanes of one warp with the
// same site); each <n_j> is a warp-wide integer sum (limb reductions),
// skipped when no lane has phonons at site j.
template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_accum(const DevModel* __restrict__ M, Counters* ctr,
                                                      const uint64_t* __restrict__ keys,
                                                      const double2* __restrict__ vec,
                                                      unsigned long long* __restrict__ part)
{
    __shared__ unsigned long long sh[kBlock / 32][kObsStride][2];
    if (ctr->err) return;
    const int N = M->N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = lane; t < 2 * N + 1; t += 32) sh[warp][t][0] = sh[warp][t][1] = 0ull;
    __syncwarp();
    const int fmt = M->fmt;
    const uint32_t q = ctr->q;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const bool uni = M->uniform_radix != 0;
    const UDiv rd0 = M->div_radix[0];
    const UDiv dexc = M->div_exc;
    int wf[W + 1];
#pragma unroll
    for (int i = 0; i <= W; ++i) wf[i] = M->word_first[i];
    unsigned long long nh = 0, nl = 0;
    for (uint64_t rb = (uint64_t)gw * 32; rb < q; rb += (uint64_t)nw * 32) {
        uint64_t row = rb + lane;
        unsigned long long hi = 0, lo = 0;
        Key<W> k;
#pragma unroll
        for (int i = 0; i < W; ++i) k.w[i] = 0;
        if (row < q) {
            if (fmt == 1) {
                double2 v = vec[row];
                double w = v.x * v.x + v.y * v.y;
                if (w != 0.0) split_weight(w, hi, lo);
            } else {
                dwf w = dw_norm2(reinterpret_cast<const float4*>(vec)[row]);
                if (w.hi != 0.0f) {
                    __int128 F = fix84(w.hi) + fix84(w.lo);
                    if (F < 0) F = 0;
                    hi = (unsigned long long)(F >> 32);
                    lo = (unsigned long long)(F & 0xFFFFFFFF);
                }
            }
            if (hi | lo) k = load_key<W>(keys, row);
        }
        bool live = (hi | lo) != 0ull;
        uint64_t q0 = udiv(k.w[0], dexc);
        int s = (int)(k.w[0] - q0 * dexc.d);
        if (live) {
            atomicAdd(&sh[warp][s][0], hi);
            atomicAdd(&sh[warp][s][1], lo);
        }
        nh += hi;
        nl += lo;
        // every phonon digit, with the divisor held in registers when all
        // sites share one radix
        auto digits = [&](auto uniform) {
#pragma unroll
            for (int wd = 0; wd < W; ++wd) {
                uint64_t x = (wd == 0) ? q0 : k.w[wd];
                for (int j = wf[wd]; j < wf[wd + 1]; ++j) {
                    UDiv dv;
                    if constexpr (decltype(uniform)::value) dv = rd0;
                    else dv = M->div_radix[j];
                    uint64_t xq = udiv(x, dv);
                    unsigned long long nj = x - xq * dv.d;
                    x = xq;
                    if (__any_sync(0xffffffffu, nj != 0ull)) {
                        unsigned long long a = warp_sum_limbs(hi * nj), c = warp_sum_limbs(lo * nj);
                        if (lane == 0) {
                            sh[warp][N + j][0] += a;
                            sh[warp][N + j][1] += c;
                        }
                    }
                }
            }
        };
        if (uni) digits(std::true_type{});
        else digits(std::false_type{});
    }
    nh = warp_sum_u64(nh);
    nl = warp_sum_u64(nl);
    if (lane == 0) {
        sh[warp][2 * N][0] += nh;
        sh[warp][2 * N][1] += nl;
    }
    __syncthreads();
    // integer sums do not depend on the order: blocks add into the totals
    for (int t = threadIdx.x; t < 2 * N + 1; t += blockDim.x) {
        unsigned long long ah = 0, al = 0;
        for (int wp = 0; wp < kBlock / 32; ++wp) {
            ah += sh[wp][t][0];
            al += sh[wp][t][1];
        }
        if (ah) atomicAdd(&part[2 * t], ah);
        if (al) atomicAdd(&part[2 * t + 1], al);
    }
}

// floor(w 2^84) = hi 2^32 + lo for 0 <= w < 2^32, from the bits of w with
// integer operations only (the same values as split_weight, whose FP64
// floor and conversions cost the FP64 pipe about four operations per row).
__device__ __forceinline__ void split_weight_int(double w, unsigned long long& hi, unsigned long long& lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(w);
    const int e = (int)((b >> 52) & 0x7FF);
    hi = lo = 0;
    if (e == 0) return;                                  // zero or below 2^-1022
    const unsigned long long m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
    const int sh = e - 991;                              // w 2^84 = m 2^sh
    unsigned __int128 v;
    if (sh >= 0) v = (unsigned __int128)m << sh;
    else if (sh > -64) v = (unsigned __int128)(m >> -sh);
    else return;
    hi = (unsigned long long)(v >> 32);
    lo = (unsigned long long)(v & 0xFFFFFFFFull);
}

// k_obs_accum for at most 16 sites and one model: the same integer sums, with
// each thread keeping its own <n_j> limbs in registers over all its rows (one
// warp reduction per site at the end instead of one per site and round of 32
// rows).  Per-thread sums cannot overflow: the hi limbs of all rows sum to at
// most 2^52 ||c||^2 K.
template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_accum16(const DevModel* __restrict__ M, Counters* ctr,
                                                        const uint64_t* __restrict__ keys,
                                                        const double2* __restrict__ vec,
                                                        unsigned long long* __restrict__ part)
{
    constexpr int NS = 16;
    __shared__ unsigned long long sh[kBlock / 32][kObsStride][2];
    if (ctr->err) return;
    const int N = M->N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = lane; t < 2 * N + 1; t += 32) sh[warp][t][0] = sh[warp][t][1] = 0ull;
    __syncwarp();
    const int fmt = M->fmt;
    const uint32_t q = ctr->q;
    const bool uni = M->uniform_radix != 0;
    const UDiv rd0 = M->div_radix[0];
    const UDiv dexc = M->div_exc;
    const bool r8 = M->r8_ok != 0;
    const uint32_t rmag = M->r_magic, rad = (uint32_t)rd0.d;
    int wf[W + 1];
#pragma unroll
    for (int i = 0; i <= W; ++i) wf[i] = M->word_first[i];
    unsigned long long ah[NS], al[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) ah[j] = al[j] = 0ull;
    unsigned long long nh = 0, nl = 0;
    // two rows per thread and round, with the amplitude and key loads of both
    // issued before any arithmetic (the key no longer waits for the weight)
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r0 = blockIdx.x * blockDim.x + threadIdx.x; r0 < q; r0 += 2 * stride) {
        float4 va[2];
        Key<W> kk[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint32_t row = r0 + (uint32_t)u * stride;      // q < 2^31: no wrap
            va[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < W; ++i) kk[u].w[i] = 0;
            if (row < q) {
                va[u] = reinterpret_cast<const float4*>(vec)[row];
                kk[u] = load_key<W>(keys, row);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            unsigned long long hi = 0, lo = 0;
            if (fmt == 1) {
                const double vx = __hiloint2double(__float_as_int(va[u].y), __float_as_int(va[u].x));
                const double vy = __hiloint2double(__float_as_int(va[u].w), __float_as_int(va[u].z));
                split_weight_int(vx * vx + vy * vy, hi, lo);
            } else {
                const dwf w = dw_norm2(va[u]);
                if (w.hi != 0.0f) {
                    __int128 F = fix84(w.hi) + fix84(w.lo);
                    if (F < 0) F = 0;
                    hi = (unsigned long long)(F >> 32);
                    lo = (unsigned long long)(F & 0xFFFFFFFF);
                }
            }
            if (!(hi | lo)) continue;                // rows past q have zero weight
            const Key<W>& k = kk[u];
            const uint64_t q0 = udiv(k.w[0], dexc);
            const int s = (int)(k.w[0] - q0 * dexc.d);
            atomicAdd(&sh[warp][s][0], hi);
            atomicAdd(&sh[warp][s][1], lo);
            nh += hi;
            nl += lo;
            if (W == 1 && r8) {
                // two independent chains of 32-bit digit divisions
                const uint64_t xh = udiv(q0, M->div_r8);
                uint32_t x0 = (uint32_t)(q0 - xh * M->div_r8.d), x1 = (uint32_t)xh;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t q0j = __umulhi(x0, rmag), q1j = __umulhi(x1, rmag);
                    const uint32_t n0 = x0 - q0j * rad, n1 = x1 - q1j * rad;
                    x0 = q0j;
                    x1 = q1j;
                    ah[j] += hi * n0;
                    al[j] += lo * n0;
                    ah[j + 8] += hi * n1;            // zero past the last site
                    al[j + 8] += lo * n1;
                }
            } else {
#pragma unroll
                for (int wd = 0; wd < W; ++wd) {
                    uint64_t x = (wd == 0) ? q0 : k.w[wd];
#pragma unroll
                    for (int j = 0; j < NS; ++j) {
                        if (j < wf[wd] || j >= wf[wd + 1]) continue;
                        const UDiv dv = uni ? rd0 : M->div_radix[j];
                        const uint64_t xq = udiv(x, dv);
                        const uint32_t nj = (uint32_t)(x - xq * dv.d);
                        x = xq;
                        ah[j] += hi * nj;
                        al[j] += lo * nj;
                    }
                }
            }
        }
    }
    nh = warp_sum_u64(nh);
    nl = warp_sum_u64(nl);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        if (j >= N) break;                   // uniform
        const unsigned long long a = warp_sum_u64(ah[j]), c = warp_sum_u64(al[j]);
        if (lane == 0) {
            sh[warp][N + j][0] += a;
            sh[warp][N + j][1] += c;
        }
    }
    if (lane == 0) {
        sh[warp][2 * N][0] += nh;
        sh[warp][2 * N][1] += nl;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * N + 1; t += blockDim.x) {
        unsigned long long ah2 = 0, al2 = 0;
        for (int wp = 0; wp < kBlock / 32; ++wp) {
            ah2 += sh[wp][t][0];
            al2 += sh[wp][t][1];
        }
        if (ah2) atomicAdd(&part[2 * t], ah2);
        if (al2) atomicAdd(&part[2 * t + 1], al2);
    }
}

// Ensembles: the same integer sums per (realisation, site), accumulated in
// shared memory when the R x 2N table fits there, else in global memory.
template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_accum_batch(const DevModel* __restrict__ M, Counters* ctr,
                                                            const uint64_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ meta,
                                                            const double2* __restrict__ vec,
                                                            unsigned long long* __restrict__ acc, int use_shared)
{
    extern __shared__ unsigned long long shb[];
    if (ctr->err) return;
    const int N = M->N, R = M->batch, L = 2 * R * N + 1;
    if (use_shared) {
        for (int t = threadIdx.x; t < 2 * L; t += blockDim.x) shb[t] = 0ull;
        __syncthreads();
    }
    unsigned long long* dst = use_shared ? shb : acc;
    const int fmt = M->fmt;
    const uint32_t q = ctr->q;
    unsigned long long nh = 0, nl = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        unsigned long long hi = 0, lo = 0;
        if (fmt == 1) {
            double2 v = vec[i];
            double w = v.x * v.x + v.y * v.y;
            if (w == 0.0) continue;
            split_weight(w, hi, lo);
        } else {
            dwf w = dw_norm2(reinterpret_cast<const float4*>(vec)[i]);
            if (w.hi == 0.0f) continue;
            __int128 F = fix84(w.hi) + fix84(w.lo);
            if (F <= 0) continue;
            hi = (unsigned long long)(F >> 32);
            lo = (unsigned long long)(F & 0xFFFFFFFF);
        }
        Key<W> k = load_key<W>(keys, i);
        int rz = key_real<W>(k, M), s = meta_s(meta[i]);
        atomicAdd(&dst[2 * (rz * N + s)], hi);
        atomicAdd(&dst[2 * (rz * N + s) + 1], lo);
        nh += hi;
        nl += lo;
        uint64_t q0 = udiv(k.w[0], M->div_exc);
#pragma unroll
        for (int wd = 0; wd < W; ++wd) {
            uint64_t x = (wd == 0) ? q0 : k.w[wd];
            for (int j = M->word_first[wd]; j < M->word_first[wd + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                unsigned long long nj = x - xq * M->div_radix[j].d;
                x = xq;
                if (nj) {
                    atomicAdd(&dst[2 * (R * N + rz * N + j)], hi * nj);
                    atomicAdd(&dst[2 * (R * N + rz * N + j) + 1], lo * nj);
                }
            }
        }
    }
    nh = warp_sum_u64(nh);
    nl = warp_sum_u64(nl);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&dst[2 * (L - 1)], nh);
        atomicAdd(&dst[2 * (L - 1) + 1], nl);
    }
    if (use_shared) {
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * L; t += blockDim.x)
            if (shb[t]) atomicAdd(&acc[t], shb[t]);
    }
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_finish_batch(const DevModel* __restrict__ M, Counters* ctr,
                                                             const uint64_t* __restrict__ table, uint64_t slots,
                                                             const uint64_t* __restrict__ psi0_keys,
                                                             const double2* __restrict__ psi0_amp, int64_t n0,
                                                             const double2* __restrict__ vec, double dt, int mode,
                                                             unsigned long long* __restrict__ acc,
                                                             double* __restrict__ obs, int rec_len)
{
    if (ctr->err) return;
    const int N = M->N, R = M->batch, L = 2 * R * N + 1;
    double* rec = obs + (size_t)ctr->rec_index * rec_len;
    __shared__ double nrm;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        unsigned long long hi = acc[2 * i], lo = acc[2 * i + 1];
        acc[2 * i] = acc[2 * i + 1] = 0ull;
        hi += lo >> 32;
        lo &= 0xFFFFFFFFull;
        double v = (double)hi * 2.220446049250313e-16 + (double)lo * 5.169878828456423e-26;
        if (i < L - 1) rec[PACES_OBS_FIXED + i] = v;
        else nrm = v;
    }
    // C_r(t) = <psi0|psi(t)> restricted to realisation r (psi(0) is replicated in blocks of n0/R)
    const int64_t per = n0 / R;
    double csum[2] = {0.0, 0.0};
    for (int rz = threadIdx.x; rz < R; rz += blockDim.x) {
        double cr = 0.0, ci = 0.0;
        for (int64_t k = (int64_t)rz * per; k < (int64_t)(rz + 1) * per; ++k) {
            Key<W> key = load_key<W>(psi0_keys, (uint64_t)k);
            int64_t r = table_lookup<W>(table, slots, key);
            if (r < 0) continue;
            double2 a = psi0_amp[k], c;
            if (M->fmt == 1) {
                c = vec[r];
            } else {
                float4 v = reinterpret_cast<const float4*>(vec)[r];
                c = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
            }
            cr += a.x * c.x + a.y * c.y;
            ci += a.x * c.y - a.y * c.x;
        }
        rec[PACES_OBS_FIXED + 2 * R * N + 2 * rz] = cr;
        rec[PACES_OBS_FIXED + 2 * R * N + 2 * rz + 1] = ci;
        csum[0] += cr;
        csum[1] += ci;
    }
    __shared__ double cs[2];
    block_sum<kBlock, 2>(csum, cs);
    if (threadIdx.x == 0) {
        bool initial = mode == 1;
        if (mode == 2) ctr->kept = ctr->q;
        double norm = nrm;
        double t = initial ? 0.0 : ctr->time + dt;
        ctr->time = t;
        ctr->rec_index += 1;
        rec[PACES_OBS_TIME] = t;
        rec[PACES_OBS_NORM] = norm;
        rec[PACES_OBS_NORM_PHI0] = initial ? norm : ctr->norm_phi0;
        rec[PACES_OBS_ENERGY] = initial ? 0.0 : ctr->energy;
        rec[PACES_OBS_C_RE] = cs[0] / R;
        rec[PACES_OBS_C_IM] = cs[1] / R;
        rec[PACES_OBS_ROWS] = (double)ctr->q;
        rec[PACES_OBS_KEPT] = (double)ctr->kept;
        rec[PACES_OBS_NNZ] = initial ? 0.0 : (double)(ctr->nnz + ctr->q);
        rec[PACES_OBS_TERMS] = initial ? 0.0 : (double)ctr->nterms;
        rec[PACES_OBS_NORM_BEFORE] = initial ? norm : ctr->norm_last;
        rec[PACES_OBS_SUBSTEPS] = initial ? 0.0 : (double)ctr->nsub;
        rec[PACES_OBS_HBOUND] = initial ? 0.0 : (double)ctr->hbound * (1.0 / 1048576.0);
        ctr->norm_last = norm;
        ctr->nnz = 0;
    }
}

// mode: 0 after a step, 1 the record of set_state, 2 after the first step
template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_finish(const DevModel* __restrict__ M, Counters* ctr,
                                                       const uint64_t* __restrict__ table, uint64_t slots,
                                                       const uint64_t* __restrict__ psi0_keys,
                                                       const double2* __restrict__ psi0_amp, int64_t n0,
                                                       const double2* __restrict__ vec, double dt, int mode,
                                                       unsigned long long* __restrict__ part,
                                                       double* __restrict__ obs, int rec_len)
{
    if (ctr->err) return;
    const int N = M->N;
    double* rec = obs + (size_t)ctr->rec_index * rec_len;
    __shared__ double nrm;
    for (int i = threadIdx.x; i < 2 * N + 1; i += blockDim.x) {
        unsigned long long hi = part[2 * i], lo = part[2 * i + 1];
        part[2 * i] = part[2 * i + 1] = 0ull;     // ready for the next pass
        // (hi + lo 2^-32) 2^-52, carrying the upper bits of lo into hi first
        hi += lo >> 32;
        lo &= 0xFFFFFFFFull;
        double acc = (double)hi * 2.220446049250313e-16 + (double)lo * 5.169878828456423e-26;
        if (i < 2 * N) rec[PACES_OBS_FIXED + i] = acc;
        else nrm = acc;
    }
    double acc[2] = {0.0, 0.0};
    for (int64_t k = threadIdx.x; k < n0; k += blockDim.x) {
        Key<W> key = load_key<W>(psi0_keys, (uint64_t)k);
        int64_t r = table_lookup<W>(table, slots, key);
        if (r < 0) continue;
        double2 a = psi0_amp[k], c;
        if (M->fmt == 1) {
            c = vec[r];
        } else {
            float4 v = reinterpret_cast<const float4*>(vec)[r];
            c = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
        }
        acc[0] += a.x * c.x + a.y * c.y;    // conj(a) * c
        acc[1] += a.x * c.y - a.y * c.x;
    }
    __shared__ double cs[2];
    block_sum<kBlock, 2>(acc, cs);
    if (threadIdx.x == 0) {
        bool initial = mode == 1;
        if (mode == 2) ctr->kept = ctr->q;      // the first step propagates every row
        double norm = nrm;                       // exact fixed-point sum of |c|^2
        double t = initial ? 0.0 : ctr->time + dt;
        ctr->time = t;
        ctr->rec_index += 1;
        rec[PACES_OBS_TIME] = t;
        rec[PACES_OBS_NORM] = norm;
        rec[PACES_OBS_NORM_PHI0] = initial ? norm : ctr->norm_phi0;
        rec[PACES_OBS_ENERGY] = initial ? 0.0 : ctr->energy;
        rec[PACES_OBS_C_RE] = cs[0];
        rec[PACES_OBS_C_IM] = cs[1];
        rec[PACES_OBS_ROWS] = (double)ctr->q;
        rec[PACES_OBS_KEPT] = (double)ctr->kept;
        rec[PACES_OBS_NNZ] = initial ? 0.0 : (double)(ctr->nnz + ctr->q);
        rec[PACES_OBS_TERMS] = initial ? 0.0 : (double)ctr->nterms;
        rec[PACES_OBS_NORM_BEFORE] = initial ? norm : ctr->norm_last;
        rec[PACES_OBS_SUBSTEPS] = initial ? 0.0 : (double)ctr->nsub;
        rec[PACES_OBS_HBOUND] = initial ? 0.0 : (double)ctr->hbound * (1.0 / 1048576.0);
        ctr->norm_last = norm;
        ctr->nnz = 0;            // the next step's P H P build counts from zero
    }
}

// Descriptors of rows given only as keys (full decode).
template <int W>
__global__ void k_meta_from_keys(const DevModel* __restrict__ M, const uint64_t* __restrict__ keys, uint32_t n,
                                 uint32_t* __restrict__ meta)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, i);
        uint64_t q0 = udiv(k.w[0], M->div_exc);
        int s = (int)(k.w[0] - q0 * M->div_exc.d), ns = 0, nph = 0;
        for (int w = 0; w < W; ++w) {
            uint64_t x = (w == 0) ? q0 : k.w[w];
            for (int j = M->word_first[w]; j < M->word_first[w + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                int nj = (int)(x - xq * M->div_radix[j].d);
                x = xq;
                nph += nj;
                if (j == s) ns = nj;
            }
        }
        meta[i] = meta_pack(s, ns, nph);
    }
}

// ---------------------------------------------------------------- export helpers
template <int W>
__global__ void k_decode(const DevModel* __restrict__ M, const uint64_t* __restrict__ keys, uint32_t n,
                         int32_t* __restrict__ site, int32_t* __restrict__ occ)
{
    const int N = M->N, C = N + (M->batch > 1 ? 1 : 0);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, i);
        uint64_t q0 = udiv(k.w[0], M->div_exc);
        site[i] = (int32_t)(k.w[0] - q0 * M->div_exc.d);
        for (int w = 0; w < W; ++w) {
            uint64_t x = (w == 0) ? q0 : k.w[w];
            for (int j = M->word_first[w]; j < M->word_first[w + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                occ[(uint64_t)i * C + j] = (int32_t)(x - xq * M->div_radix[j].d);
                x = xq;
            }
        }
        if (C > N) occ[(uint64_t)i * C + N] = key_real<W>(k, M);
    }
}

__global__ void k_export_csr(const DevModel* __restrict__ M, uint32_t q, const uint64_t* __restrict__ off,
                             const uint32_t* __restrict__ col, const uint8_t* __restrict__ cidv,
                             const uint8_t* __restrict__ cnt, int32_t* __restrict__ cols, double* __restrict__ vals)
{
    int P = M->P;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        uint64_t o = off[i];
        for (int e = 0; e < cnt[i]; ++e) {
            cols[o + e] = (int32_t)col[(uint64_t)i * P + e];
            vals[o + e] = M->coef[cidv[(uint64_t)i * P + e]];
        }
    }
}

// ---------------------------------------------------------------- launchers
template <int W>
static int trunc_w(const Bufs& b, int gin, int gout, double th2, int step, cudaStream_t st, bool counted = false)
{
    if (!counted)
        k_trunc_count<<<b.G, kBlock, 0, st>>>(b.V[0], b.ctr, th2, dw_from_double(th2), b.fmt, b.keepw, b.blk_cnt);
    k_scan<<<1, 1024, 0, st>>>(b.blk_cnt, b.blk_off, b.G, b.ctr, kScanTrunc, 0, b.cap_rows, step);
    int n = launch_sorted_m(b, gin, gout, step, st);
    return n < 0 ? n : n + (counted ? 1 : 2);
}

template <int W>
static int level_w(const Bufs& b, int gen, int f, int rescue_gen, int step, cudaStream_t st)
{
    k_level_insert<W><<<b.grid, kBlock, 0, st>>>(b.model, b.ctr, f, b.keys[gen], b.meta[gen], b.table[gen],
                                                 b.table_slots,
                                                 b.cand_slot, b.cand_cap, step);
    k_level_flags<W><<<b.G, kBlock, 0, st>>>(b.model, b.ctr, f, b.table[gen], b.cand_slot,
                                             reinterpret_cast<uint32_t*>(b.masks), b.blk_cnt);
    k_scan<<<1, 1024, 0, st>>>(b.blk_cnt, b.blk_off, b.G, b.ctr, kScanLevel, f, b.cap_rows, step);
    const uint64_t* ot = rescue_gen >= 0 ? b.table[rescue_gen] : nullptr;
    k_level_scatter<W><<<b.G, kBlock, 0, st>>>(b.model, b.ctr, f, b.keys[gen], b.meta[gen], b.table[gen],
                                               b.cand_slot, reinterpret_cast<const uint32_t*>(b.masks), b.blk_off);
    k_level_rescue<W><<<b.grid, kBlock, 0, st>>>(b.ctr, f, b.keys[gen], ot, b.table_slots, b.V[0], b.V[1], b.from);
    return 5;
}

template <int W>
static int csr_w(const Bufs& b, int gen, cudaStream_t st)
{
#define PACES_CSR_ARGS \
    b.model, b.ctr, b.keys[gen], b.meta[gen], b.table[gen], b.table_slots, b.cand_slot, b.col, b.cid, b.cnt, \
        b.diag
    // the row bound is a maximum over this build's rows only
    cudaMemsetAsync(reinterpret_cast<char*>(b.ctr) + offsetof(Counters, hbound), 0, sizeof(unsigned long long), st);
    // one-word keys: one thread per row (the per-row key images fit in registers)
    if (W == 1 && b.D <= 4) k_csr_row<1, 4><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
    else if (W == 1 && b.D <= 8) k_csr_row<1, 8><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
    else if (b.D <= 4) k_csr_grp<W, 4><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
    else if (b.D <= 8) k_csr_grp<W, 8><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
    else if (b.D <= 16) k_csr_grp<W, 16><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
    else if (b.D <= 32) k_csr_grp<W, 32><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
    else k_csr<W><<<b.grid, kBlock, 0, st>>>(PACES_CSR_ARGS);
#undef PACES_CSR_ARGS
    return 1;
}

template <int W>
static int observe_w(const Bufs& b, int gen, const double2* vec, double dt, int mode, cudaStream_t st)
{
    if (b.batch > 1) {
        size_t shm = sizeof(unsigned long long) * 2 * (size_t)(2 * b.batch * b.N + 1);
        int use_shared = shm <= kObsSharedMax;
        k_obs_accum_batch<W><<<b.G, kBlock, use_shared ? shm : 0, st>>>(b.model, b.ctr, b.keys[gen], b.meta[gen], vec,
                                                                        b.obs_part, use_shared);
        k_obs_finish_batch<W><<<1, kBlock, 0, st>>>(b.model, b.ctr, b.table[gen], b.table_slots, b.psi0_keys,
                                                    b.psi0_amp, b.n0, vec, dt, mode, b.obs_part, b.obs, b.rec_len);
        return 2;
    }
    if (b.N <= 16) k_obs_accum16<W><<<b.G, kBlock, 0, st>>>(b.model, b.ctr, b.keys[gen], vec, b.obs_part);
    else k_obs_accum<W><<<b.G, kBlock, 0, st>>>(b.model, b.ctr, b.keys[gen], vec, b.obs_part);
    k_obs_finish<W><<<1, kBlock, 0, st>>>(b.model, b.ctr, b.table[gen], b.table_slots, b.psi0_keys, b.psi0_amp,
                                          b.n0, vec, dt, mode, b.obs_part, b.obs, b.rec_len);
    return 2;
}

template <int W>
static int prepare_w(const Bufs& b)
{
    size_t shm = sizeof(unsigned long long) * 2 * (size_t)(2 * b.batch * b.N + 1);
    if (b.batch > 1 && shm <= kObsSharedMax)
        cudaFuncSetAttribute(k_obs_accum_batch<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    return 0;
}

#define PACES_DISPATCH_W(W_, CALL)                                                      \
    switch (W_) {                                                                        \
    case 1: { constexpr int KW = 1; return CALL; }                                       \
    case 2: { constexpr int KW = 2; return CALL; }                                       \
    case 3: { constexpr int KW = 3; return CALL; }                                       \
    case 4: { constexpr int KW = 4; return CALL; }                                       \
    default: return -1;                                                                  \
    }

int launch_insert_rows(const Bufs& b, int gen, uint32_t n, cudaStream_t st)
{
    int grid = b.grid;
    PACES_DISPATCH_W(b.W, (k_insert_rows<KW><<<grid, kBlock, 0, st>>>(b.keys[gen], n, b.table[gen], b.table_slots,
                                                                       b.ctr), 1))
}

int launch_truncate(const Bufs& b, int gin, int gout, double th2, int step, cudaStream_t st)
{
    PACES_DISPATCH_W(b.W, trunc_w<KW>(b, gin, gout, th2, step, st))
}

int launch_truncate_nom(const Bufs& b, int gin, int gout, uint64_t q_nom, uint64_t seed, int step, cudaStream_t st)
{
    int n = launch_topq_select(b, gin, q_nom, seed, st);
    if (n < 0) return n;
    PACES_DISPATCH_W(b.W, n - 1 + trunc_w<KW>(b, gin, gout, 0.0, step, st, true))
}

int launch_level(const Bufs& b, int gen, int f, int rescue_gen, int step, cudaStream_t st)
{
    PACES_DISPATCH_W(b.W, level_w<KW>(b, gen, f, rescue_gen, step, st))
}

int launch_csr(const Bufs& b, int gen, cudaStream_t st) { PACES_DISPATCH_W(b.W, csr_w<KW>(b, gen, st)) }

int launch_observe(const Bufs& b, int gen, const double2* vec, double dt, int mode, cudaStream_t st)
{
    PACES_DISPATCH_W(b.W, observe_w<KW>(b, gen, vec, dt, mode, st))
}

int prepare_kernels(const Bufs& b) { PACES_DISPATCH_W(b.W, prepare_w<KW>(b)) }

int launch_decode(const Bufs& b, int gen, uint32_t n, int32_t* site, int32_t* occ, cudaStream_t st)
{
    int grid = b.grid;
    PACES_DISPATCH_W(b.W, (k_decode<KW><<<grid, kBlock, 0, st>>>(b.model, b.keys[gen], n, site, occ), 1))
}

int launch_meta_from_keys(const Bufs& b, int gen, uint32_t n, cudaStream_t st)
{
    int grid = b.grid;
    PACES_DISPATCH_W(b.W, (k_meta_from_keys<KW><<<grid, kBlock, 0, st>>>(b.model, b.keys[gen], n, b.meta[gen]), 1))
}

int launch_export_csr(const Bufs& b, uint32_t q, const uint64_t* off, int32_t* cols, double* vals, cudaStream_t st)
{
    k_export_csr<<<b.grid, kBlock, 0, st>>>(b.model, q, off, b.col, b.cid, b.cnt, cols, vals);
    return 1;
}

}  // namespace paces
