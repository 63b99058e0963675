// kern_topq.cu -- truncation to the q_nom heaviest rows, the paper's own
// scheme (Sec. "Truncation & post-adaptation detruncation"; App. "How to
// weight states for truncation"), as a device-side radix select: no host
// round trip, so the step stays one captured graph.
//
// Each row gets a selection key (w, tk), larger first, compared in that order:
//   w   |c|^2 as FP64 bits (non-negative doubles order like their bit
//       patterns).  FP64 storage: both products and the sum rounded
//       separately, as threshold truncation evaluates them; double-word
//       storage: hi + lo of the double-word |c|^2, exact in FP64.
//   tk  (u with its low 32 bits cleared) | (0xFFFFFFFF - row), where u is the
//       tie hash of (seed, t, s, n_0 .. n_{N-1}): z = seed + G t, then
//       z = mix(z xor v) for every entry v, mix the output function of
//       SplitMix64 (Steele, Lea & Flood 2014), G = 0x9E3779B97F4A7C15, and t
//       the index of the observables record the step writes.  The appendix
//       asks for degenerate weights at the cutoff to be ordered at random; tk
//       does that and, holding the row, is unique, so exactly q_nom rows are
//       kept whenever q > q_nom.
// Weights are selected first: five passes of 12 bits and one of 4, each a
// histogram of the rows whose higher bits match the prefix chosen so far,
// then a one-block pick of the digit at which the running count (from the
// top) reaches the rank still to place.  Only when more rows share the cut
// weight than places remain are their tie keys computed and selected the
// same way.  The keep bits and chunk counts are written as threshold
// truncation writes them, so the compaction kernels are shared.
#include "runtime.h"

namespace paces {

namespace {

constexpr int kSelBits = 12;
constexpr int kSelBins = 1 << kSelBits;
constexpr int kSelPasses = 6;                  // 5 x 12 + 4 = 64 bits
constexpr int kSelBlock = 256;

__device__ __forceinline__ int pass_shift(int p) { return p < 5 ? 52 - 12 * p : 0; }
__device__ __forceinline__ int pass_bits(int p) { return p < 5 ? 12 : 4; }

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t weight_bits(const double2* c, uint64_t i, int fmt)
{
    double w;
    if (fmt == 1) {
        double2 v = c[i];
        w = __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
    } else {
        dwf d = dw_norm2(reinterpret_cast<const float4*>(c)[i]);
        w = (double)d.hi + (double)d.lo;
    }
    if (!(w > 0.0)) w = 0.0;                  // -0 and NaN order as 0
    return (uint64_t)__double_as_longlong(w);
}

}  // namespace

// Weight bits of every row; resets the selection state.
__global__ void __launch_bounds__(kSelBlock) k_topq_prep(const double2* __restrict__ c, Counters* ctr, int fmt,
                                                          uint64_t q_nom, TopqState* st,
                                                          uint64_t* __restrict__ wk)
{
    if (ctr->err) return;
    const uint32_t q = ctr->q;
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < kSelBins; t += blockDim.x) st->hist[t] = 0u;
        if (threadIdx.x == 0) {
            st->all = (uint64_t)q <= q_nom ? 1u : 0u;
            st->phase = 0u;
            st->ties_all = 0u;
            st->prefix = 0ull;
            st->krem = q_nom;
            st->w_cut = 0ull;
            st->tk_cut = 0ull;
        }
    }
    if ((uint64_t)q <= q_nom) return;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x)
        wk[i] = weight_bits(c, i, fmt);
}

// Histogram of the next digit of the rows still in the running.
__global__ void __launch_bounds__(kSelBlock) k_topq_hist(const Counters* __restrict__ ctr, TopqState* st,
                                                          const uint64_t* __restrict__ wk,
                                                          const uint64_t* __restrict__ tk, int phase, int pass)
{
    __shared__ uint32_t h[kSelBins];
    if (ctr->err || st->all || st->phase != (uint32_t)phase) return;
    for (int t = threadIdx.x; t < kSelBins; t += blockDim.x) h[t] = 0u;
    __syncthreads();
    const uint32_t q = ctr->q;
    const int shift = pass_shift(pass), bits = pass_bits(pass);
    const int hs = shift + bits;                               // bits above this digit
    const uint64_t prefix = st->prefix, w_cut = st->w_cut;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t key;
        if (phase == 0) {
            key = wk[i];
        } else {
            if (wk[i] != w_cut) continue;
            key = tk[i];
        }
        if (hs < 64 && (key >> hs) != (prefix >> hs)) continue;
        atomicAdd(&h[(key >> shift) & ((1u << bits) - 1u)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (1 << bits); t += blockDim.x)
        if (h[t]) atomicAdd(&st->hist[t], h[t]);
}

// One block: the digit at which the count from the top reaches the rank.
__global__ void __launch_bounds__(1024) k_topq_pick(const Counters* __restrict__ ctr, TopqState* st, int phase,
                                                    int pass)
{
    __shared__ uint32_t sel_d, sel_n;
    __shared__ unsigned long long sel_above;
    if (ctr->err || st->all || st->phase != (uint32_t)phase) return;
    if (threadIdx.x == 0) {
        sel_d = 0u;
        sel_n = 0u;
        sel_above = 0ull;
    }
    const int shift = pass_shift(pass), bits = pass_bits(pass), nb = 1 << bits;
    // thread t owns bins nb-1-4t .. nb-4-4t (descending)
    uint32_t own[4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int b = nb - 1 - (4 * (int)threadIdx.x + k);
        own[k] = b >= 0 ? st->hist[b] : 0u;
        s += own[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<1024>(s, &tot);
    const unsigned long long krem = st->krem;
    unsigned long long run = ex;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int b = nb - 1 - (4 * (int)threadIdx.x + k);
        if (b >= 0 && run < krem && run + own[k] >= krem) {
            sel_d = (uint32_t)b;
            sel_n = own[k];
            sel_above = run;
        }
        run += own[k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kSelBins; t += blockDim.x) st->hist[t] = 0u;
    if (threadIdx.x == 0) {
        st->prefix |= (unsigned long long)sel_d << shift;
        st->krem = krem - sel_above;
        if (pass == kSelPasses - 1) {
            if (phase == 0) {
                st->w_cut = st->prefix;
                st->prefix = 0ull;
                if (sel_n == st->krem) {              // every row of the cut weight fits
                    st->ties_all = 1u;
                    st->phase = 2u;
                } else {
                    st->phase = 1u;
                }
            } else {
                st->tk_cut = st->prefix;
                st->phase = 2u;
            }
        }
    }
}

// Tie keys of the rows that share the cut weight (phase 1 only).
template <int W>
__global__ void __launch_bounds__(kSelBlock) k_topq_ties(const DevModel* __restrict__ M, const Counters* __restrict__ ctr,
                                                          TopqState* st, const uint64_t* __restrict__ keys,
                                                          const uint64_t* __restrict__ wk, uint64_t* __restrict__ tk,
                                                          uint64_t seed)
{
    if (ctr->err || st->all || st->phase != 1u) return;
    const uint32_t q = ctr->q;
    const uint64_t w_cut = st->w_cut;
    const uint64_t z0 = seed + 0x9E3779B97F4A7C15ull * (uint64_t)ctr->rec_index;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x) {
        if (wk[i] != w_cut) continue;
        Key<W> k = load_key<W>(keys, i);
        uint64_t q0 = udiv(k.w[0], M->div_exc);
        uint64_t z = mix64(z0 ^ (k.w[0] - q0 * M->div_exc.d));      // s
#pragma unroll
        for (int wd = 0; wd < W; ++wd) {
            uint64_t x = (wd == 0) ? q0 : k.w[wd];
            for (int j = M->word_first[wd]; j < M->word_first[wd + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                z = mix64(z ^ (x - xq * M->div_radix[j].d));         // n_j
                x = xq;
            }
        }
        tk[i] = (z & 0xFFFFFFFF00000000ull) | (0xFFFFFFFFull - (uint64_t)i);
    }
}

// Keep bits (32 per word) and kept rows per chunk, as threshold truncation.
__global__ void __launch_bounds__(kBlock) k_topq_keep(const Counters* __restrict__ ctr, const TopqState* __restrict__ st,
                                                      const uint64_t* __restrict__ wk, const uint64_t* __restrict__ tk,
                                                      uint32_t* __restrict__ keepw, uint32_t* __restrict__ blk_cnt)
{
    if (ctr->err) return;
    uint32_t q = ctr->q, lo, hi;
    chunk_of(q, gridDim.x, blockIdx.x, lo, hi);
    const bool all = st->all != 0u, ties_all = st->ties_all != 0u;
    const uint64_t w_cut = st->w_cut, tk_cut = st->tk_cut;
    uint32_t cnt = 0;
    for (uint32_t base = lo; base < hi; base += kBlock) {
        uint32_t i = base + threadIdx.x;
        bool keep = false;
        if (i < hi) {
            if (all) {
                keep = true;
            } else {
                uint64_t w = wk[i];
                keep = w > w_cut || (w == w_cut && (ties_all || tk[i] >= tk_cut));
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        uint32_t w0 = base + (threadIdx.x & ~31u);
        if ((threadIdx.x & 31) == 0 && w0 < hi) keepw[w0 >> 5] = bal;
        cnt += keep ? 1u : 0u;
    }
    uint32_t tot;
    block_excl_scan<kBlock>(cnt, &tot);
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = tot;
}

int launch_topq_select(const Bufs& b, int gin, uint64_t q_nom, uint64_t seed, cudaStream_t st)
{
    uint64_t* wk = reinterpret_cast<uint64_t*>(b.V[2]);
    uint64_t* tk = reinterpret_cast<uint64_t*>(b.V[3]);
    int n = 0;
    k_topq_prep<<<b.grid, kSelBlock, 0, st>>>(b.V[0], b.ctr, b.fmt, q_nom, b.topq, wk);
    ++n;
    for (int phase = 0; phase < 2; ++phase) {
        if (phase == 1) {
            switch (b.W) {
            case 1: k_topq_ties<1><<<b.grid, kSelBlock, 0, st>>>(b.model, b.ctr, b.topq, b.keys[gin], wk, tk, seed); break;
            case 2: k_topq_ties<2><<<b.grid, kSelBlock, 0, st>>>(b.model, b.ctr, b.topq, b.keys[gin], wk, tk, seed); break;
            case 3: k_topq_ties<3><<<b.grid, kSelBlock, 0, st>>>(b.model, b.ctr, b.topq, b.keys[gin], wk, tk, seed); break;
            case 4: k_topq_ties<4><<<b.grid, kSelBlock, 0, st>>>(b.model, b.ctr, b.topq, b.keys[gin], wk, tk, seed); break;
            default: return -1;
            }
            ++n;
        }
        for (int p = 0; p < kSelPasses; ++p) {
            k_topq_hist<<<b.grid, kSelBlock, 0, st>>>(b.ctr, b.topq, wk, tk, phase, p);
            k_topq_pick<<<1, 1024, 0, st>>>(b.ctr, b.topq, phase, p);
            n += 2;
        }
    }
    k_topq_keep<<<b.G, kBlock, 0, st>>>(b.ctr, b.topq, wk, tk, b.keepw, b.blk_cnt);
    return n + 1;
}

}  // namespace paces
