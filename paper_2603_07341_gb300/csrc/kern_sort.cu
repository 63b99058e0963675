// kern_sort.cu -- the kept set M in ascending basis order.
//
// After truncation the kept rows are compacted as (key, source row) pairs,
// sorted by key with a stable least-significant-digit radix sort (8-bit
// digits, only over the bits the key layout uses), and placed: keys, row
// descriptors and amplitudes gathered from their source rows, and each row
// inserted into the fresh table.  Ascending key order is ascending basis
// order -- n_{N-1} most significant, down to n_0, then the exciton site --
// the order of a sorted key array, which the paper's index matching between
// successive effective spaces by sorting and searching works on (Sec. "Formal
// operator representation and notes on parallelization").  States that
// differ by an exciton hop are then neighbours
// in M, and the regrown levels inherit that grouping from their parents, so
// the propagator's gathers of neighbour amplitudes hit cache lines that are
// already loaded.
#include "runtime.h"

namespace paces {

namespace {
constexpr int kDigits = 256;
}

// Kept rows as (key, source row) in row order (the scan of the keep bits).
// Each thread takes four consecutive rows per block scan (chunks start at
// multiples of kBlock, so the four keep bits share one 32-bit word) and issues
// the key loads of its kept rows before the scan.
template <int W>
__global__ void __launch_bounds__(kBlock) k_trunc_compact(const uint64_t* __restrict__ keys_in, Counters* ctr,
                                                          const uint32_t* __restrict__ keepw,
                                                          const uint32_t* __restrict__ blk_off,
                                                          uint64_t* __restrict__ sk, uint32_t* __restrict__ si)
{
    constexpr int kRPT = 4;
    if (ctr->err) return;
    uint32_t q = ctr->q_in, lo, hi;
    chunk_of(q, gridDim.x, blockIdx.x, lo, hi);
    uint32_t run = blk_off[blockIdx.x];
    for (uint32_t base = lo; base < hi; base += kBlock * kRPT) {
        const uint32_t i0 = base + kRPT * threadIdx.x;
        unsigned bits = 0;
        if (i0 < hi) {
            bits = (keepw[i0 >> 5] >> (i0 & 31u)) & 0xFu;
            if (hi - i0 < (uint32_t)kRPT) bits &= (1u << (hi - i0)) - 1u;
        }
        Key<W> k[kRPT];
#pragma unroll
        for (int u = 0; u < kRPT; ++u)
            if ((bits >> u) & 1u) k[u] = load_key<W>(keys_in, i0 + u);
        uint32_t tot;
        uint32_t o = run + block_excl_scan<kBlock>((uint32_t)__popc(bits), &tot);
#pragma unroll
        for (int u = 0; u < kRPT; ++u)
            if ((bits >> u) & 1u) {
                store_key<W>(sk, o, k[u]);
                si[o] = i0 + u;
                ++o;
            }
        run += tot;
    }
}

// Digit counts of each block's chunk: hist[d * G + block].
template <int W>
__global__ void __launch_bounds__(kBlock) k_rs_hist(const Counters* __restrict__ ctr, const uint64_t* __restrict__ sk,
                                                    int word, int shift, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[kDigits];
    if (ctr->err) return;
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) h[d] = 0u;
    __syncthreads();
    uint32_t n = ctr->kept, lo, hi;
    chunk_of(n, gridDim.x, blockIdx.x, lo, hi);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        atomicAdd(&h[(sk[(uint64_t)i * W + word] >> shift) & (kDigits - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) hist[(size_t)d * gridDim.x + blockIdx.x] = h[d];
}

// One block per digit d: exclusive scan of the G block counts hist[d G ..
// d G + G) in place (G <= 1024, one count per thread) and the digit's total in
// dtot[d].  The scatter adds the exclusive scan of the 256 totals itself.
__global__ void __launch_bounds__(1024) k_rs_scan(const Counters* __restrict__ ctr, uint32_t* __restrict__ hist,
                                                  uint32_t* __restrict__ dtot, int G)
{
    if (ctr->err) return;
    uint32_t* h = hist + (size_t)blockIdx.x * G;
    const uint32_t v = (int)threadIdx.x < G ? h[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan<1024>(v, &tot);
    if ((int)threadIdx.x < G) h[threadIdx.x] = ex;
    if (threadIdx.x == 0) dtot[blockIdx.x] = tot;
}

// Stable scatter of one digit.  Each block walks its chunk in tiles of
// kBlock * IPT items (IPT rounds of one item per thread, in index order).  The
// rank of an item among the equal digits of its tile is its rank in its warp
// (match) plus the counts of the earlier warps of its round plus those of the
// earlier rounds.  The tile is then staged in shared memory in digit order and
// written out so that consecutive threads write consecutive positions of one
// digit's run (coalesced), at the block's running offset of that digit.
template <int W>
struct ScatterTile {
    static constexpr int kIPT = W <= 2 ? 4 : 2;
    static constexpr int kItems = kBlock * kIPT;
};

template <int W>
__global__ void __launch_bounds__(kBlock) k_rs_scatter(const Counters* __restrict__ ctr,
                                                       const uint64_t* __restrict__ kin, const uint32_t* __restrict__ iin,
                                                       uint64_t* __restrict__ kout, uint32_t* __restrict__ iout,
                                                       int word, int shift, const uint32_t* __restrict__ offs,
                                                       const uint32_t* __restrict__ dtot)
{
    static_assert(kBlock == kDigits, "one thread per digit in the per-tile scans");
    constexpr int IPT = ScatterTile<W>::kIPT, T = ScatterTile<W>::kItems;
    __shared__ uint32_t base[kDigits];            // block's next output position per digit
    __shared__ uint32_t run[kDigits];             // items of the current tile per digit so far
    __shared__ uint32_t tstart[kDigits];          // first staged slot of each digit in the tile
    __shared__ uint32_t wc[kBlock / 32][kDigits];
    __shared__ uint64_t skey[T * W];
    __shared__ uint32_t sidx[T];
    __shared__ uint16_t sdig[T];
    if (ctr->err) return;
    uint32_t n = ctr->kept, lo, hi;
    chunk_of(n, gridDim.x, blockIdx.x, lo, hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {   // first output position of (digit, block): the digits below it, then the earlier blocks
        uint32_t all;
        const uint32_t below = block_excl_scan<kBlock>(dtot[threadIdx.x], &all);
        base[threadIdx.x] = below + offs[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
    }
    for (uint32_t t0 = lo; t0 < hi; t0 += T) {
        run[threadIdx.x] = 0u;
        int dg[IPT];
        uint32_t rk[IPT];
        Key<W> ks[IPT];
        uint32_t is[IPT];
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
#pragma unroll
            for (int w = 0; w < kBlock / 32; ++w) wc[w][threadIdx.x] = 0u;
            __syncthreads();
            const uint32_t i = t0 + (uint32_t)r * kBlock + threadIdx.x;
            const bool valid = i < hi;
#pragma unroll
            for (int x = 0; x < W; ++x) ks[r].w[x] = 0;
            is[r] = 0u;
            int d = kDigits;                      // invalid lanes match only each other
            if (valid) {
                ks[r] = load_key<W>(kin, i);
                is[r] = iin[i];
                d = (int)((kin[(uint64_t)i * W + word] >> shift) & (kDigits - 1));
            }
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t wrank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
            if (valid && wrank == 0) wc[warp][d] = (uint32_t)__popc(peers);
            __syncthreads();
            {   // exclusive prefix over the warps of this round, after the earlier rounds
                const int dd = threadIdx.x;
                uint32_t acc = run[dd];
#pragma unroll
                for (int w = 0; w < kBlock / 32; ++w) {
                    uint32_t c = wc[w][dd];
                    wc[w][dd] = acc;
                    acc += c;
                }
                run[dd] = acc;
            }
            __syncthreads();
            dg[r] = d;
            rk[r] = valid ? wc[warp][d] + wrank : 0u;
            __syncthreads();                      // wc is cleared for the next round
        }
        // first staged slot of every digit: exclusive scan of the tile counts
        uint32_t tot;
        const uint32_t st = block_excl_scan<kBlock>(run[threadIdx.x], &tot);
        tstart[threadIdx.x] = st;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            if (dg[r] < kDigits) {
                const uint32_t l = tstart[dg[r]] + rk[r];
                store_key<W>(skey, l, ks[r]);
                sidx[l] = is[r];
                sdig[l] = (uint16_t)dg[r];
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < tot; j += kBlock) {
            const int d = sdig[j];
            const uint32_t pos = base[d] + (j - tstart[d]);
            store_key<W>(kout, pos, load_key<W>(skey, j));
            iout[pos] = sidx[j];
        }
        __syncthreads();
        base[threadIdx.x] += run[threadIdx.x];
        __syncthreads();
    }
}

// Sorted M in place: keys, descriptors and amplitudes from the source rows,
// rescue map, and the fresh table.
template <int W>
__global__ void __launch_bounds__(kBlock) k_trunc_place(Counters* ctr, const uint64_t* __restrict__ sk,
                                                        const uint32_t* __restrict__ si,
                                                        const double2* __restrict__ c_in,
                                                        const uint32_t* __restrict__ meta_in,
                                                        uint64_t* __restrict__ keys_out, double2* __restrict__ c_out,
                                                        uint32_t* __restrict__ meta_out, uint64_t* table_out,
                                                        uint64_t slots, uint32_t* __restrict__ from, int step)
{
    if (ctr->err) return;
    const uint32_t n = ctr->kept;
    if constexpr (W == 1) {
        // one-word keys: kRPT rows per thread, their gathers issued together
        // and their (unique) keys inserted in warp-wide lockstep rounds: every
        // round claims, with one 16-byte compare-and-swap each, the empty
        // slots the unplaced keys stand on and loads the next slot of the
        // others.  Every lane of a warp runs the same number of rounds.
        constexpr int kRPT = 4;
        const uint32_t stride = gridDim.x * blockDim.x;
        for (uint32_t dw = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); dw < n; dw += stride * kRPT) {
            const uint32_t d0 = dw + (threadIdx.x & 31u);
            uint64_t key[kRPT], tag[kRPT];
            uint32_t pos[kRPT];
            unsigned act = 0;
#pragma unroll
            for (int k = 0; k < kRPT; ++k) {
                const uint32_t dst = d0 + (uint32_t)k * stride;
                key[k] = 0;
                tag[k] = 0;
                pos[k] = 0;
                if (dst < n) {
                    const uint32_t src = si[dst];
                    key[k] = sk[dst];
                    keys_out[dst] = key[k];
                    c_out[dst] = c_in[src];
                    meta_out[dst] = meta_in[src];
                    if (from) from[dst] = src;
                    const uint64_t h = key_hash<1>(Key<1>{{key[k]}});
                    tag[k] = ((uint64_t)fingerprint<1>(h) << 32) | dst;
                    pos[k] = (uint32_t)slot_home(h, slots);
                    act |= 1u << k;
                }
            }
            uint64_t cur[kRPT];
#pragma unroll
            for (int k = 0; k < kRPT; ++k)
                cur[k] = ((act >> k) & 1u) ? __ldcg(table_out + (uint64_t)pos[k] * 2) : 0ull;
            for (uint32_t round = 0; round <= kMaxProbe && __any_sync(0xffffffffu, act != 0); ++round) {
                unsigned emp = 0;
#pragma unroll
                for (int k = 0; k < kRPT; ++k) {    // occupied: the next slots, in flight with the claims
                    if (!((act >> k) & 1u)) continue;
                    if (cur[k] == kEmpty) {
                        emp |= 1u << k;
                    } else {
                        pos[k] = (uint32_t)slot_next(pos[k], slots);
                        cur[k] = __ldcg(table_out + (uint64_t)pos[k] * 2);
                    }
                }
#pragma unroll
                for (int k = 0; k < kRPT; ++k)      // claims, all in flight
                    if ((emp >> k) & 1u) {
                        uint64_t olo, ohi;
                        cas128(table_out + (uint64_t)pos[k] * 2, kEmpty, kEmpty, tag[k], key[k], olo, ohi);
                        if (olo == kEmpty) act &= ~(1u << k);
                        cur[k] = olo;               // lost: moves on in the next round
                    }
            }
            if (act) set_err(ctr, kErrProbe, step, 1);
        }
    } else {
        for (uint32_t dst = blockIdx.x * blockDim.x + threadIdx.x; dst < n; dst += gridDim.x * blockDim.x) {
            const uint32_t src = si[dst];
            Key<W> k = load_key<W>(sk, dst);
            store_key<W>(keys_out, dst, k);
            c_out[dst] = c_in[src];
            meta_out[dst] = meta_in[src];
            if (from) from[dst] = src;
            if (!table_insert_unique<W>(table_out, slots, k, dst)) set_err(ctr, kErrProbe, step, 1);
        }
    }
}

template <int W>
static int sorted_m(const Bufs& b, int gin, int gout, int step, cudaStream_t st)
{
    int n = 0;
    k_trunc_compact<W><<<b.G, kBlock, 0, st>>>(b.keys[gin], b.ctr, b.keepw, b.blk_off, b.sortk[0], b.sorti[0]);
    ++n;
    int cur = 0;
    for (int w = 0; w < W; ++w) {
        for (int s = 0; s < b.key_bits[w]; s += 8) {
            k_rs_hist<W><<<b.G, kBlock, 0, st>>>(b.ctr, b.sortk[cur], w, s, b.rs_hist);
            k_rs_scan<<<kDigits, 1024, 0, st>>>(b.ctr, b.rs_hist, b.rs_hist + (size_t)kDigits * b.G, b.G);
            k_rs_scatter<W><<<b.G, kBlock, 0, st>>>(b.ctr, b.sortk[cur], b.sorti[cur], b.sortk[1 - cur],
                                                     b.sorti[1 - cur], w, s, b.rs_hist,
                                                     b.rs_hist + (size_t)kDigits * b.G);
            cur = 1 - cur;
            n += 3;
        }
    }
    k_trunc_place<W><<<b.grid, kBlock, 0, st>>>(b.ctr, b.sortk[cur], b.sorti[cur], b.V[0], b.meta[gin], b.keys[gout],
                                                 b.V[1], b.meta[gout], b.table[gout], b.table_slots, b.from, step);
    return n + 1;
}

int launch_sorted_m(const Bufs& b, int gin, int gout, int step, cudaStream_t st)
{
    switch (b.W) {
    case 1: return sorted_m<1>(b, gin, gout, step, st);
    case 2: return sorted_m<2>(b, gin, gout, step, st);
    case 3: return sorted_m<3>(b, gin, gout, step, st);
    case 4: return sorted_m<4>(b, gin, gout, step, st);
    default: return -1;
    }
}

}  // namespace paces
