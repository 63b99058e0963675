// kern_step.cu -- the integer/gather stages of one time step (sm_103a):
//   a1 truncation Q (threshold, stable compaction, insertion of M into a fresh table),
//   a2/a3 one BFS level of H_eff: expansion of the frontier through H's moves,
//         hash de-duplication with first-occurrence winners, compaction,
//   a4 rescue of re-admitted amplitudes from the previous step's table,
//   a5 the restricted Hamiltonian P_m H P_m, row-pitched,
//   a7 observables.
// Paper: Sec. 3.3 (neighbour sets, Eqs. def_neighbor/def_neighbor_k/H_eff;
// truncation and post-adaptation detruncation; generating the effective
// Hamiltonian) and Sec. 3.4 (the step map).
#include "runtime.h"
#include "paces.h"

namespace paces {

// Contiguous chunk of [0, n) for block b of G, aligned to the block size so
// that 32-row bitmask words never straddle chunks.
__device__ __forceinline__ void chunk_of(uint32_t n, uint32_t G, uint32_t b, uint32_t& lo, uint32_t& hi)
{
    uint32_t c = (n + G - 1) / G;
    c = (c + kBlock - 1) / kBlock * kBlock;
    uint64_t l = (uint64_t)b * c;
    lo = (uint32_t)(l < n ? l : n);
    uint64_t h = l + c;
    hi = (uint32_t)(h < n ? h : n);
}

__device__ __forceinline__ void set_err(Counters* ctr, int code, int step, int info)
{
    if (atomicCAS(&ctr->err, 0, code) == 0) {
        ctr->err_step = step;
        ctr->err_info = info;
    }
}

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
// keep_i = re^2 + im^2 >= theta^2 in FP64 with every product and sum rounded
// separately (no FMA contraction), as the oracle evaluates it.
__global__ void __launch_bounds__(kBlock) k_trunc_count(const double2* __restrict__ c, Counters* ctr, double th2,
                                                        uint32_t* __restrict__ keepw, uint32_t* __restrict__ blk_cnt)
{
    if (ctr->err) return;
    uint32_t q = ctr->q, lo, hi;
    chunk_of(q, gridDim.x, blockIdx.x, lo, hi);
    uint32_t cnt = 0;
    for (uint32_t base = lo; base < hi; base += kBlock) {
        uint32_t i = base + threadIdx.x;
        bool keep = false;
        if (i < hi) {
            double2 v = c[i];
            keep = __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)) >= th2;
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

template <int W>
__global__ void __launch_bounds__(kBlock) k_trunc_scatter(const uint64_t* __restrict__ keys_in,
                                                          const double2* __restrict__ c_in, Counters* ctr,
                                                          const uint32_t* __restrict__ keepw,
                                                          const uint32_t* __restrict__ blk_off,
                                                          uint64_t* __restrict__ keys_out, double2* __restrict__ c_out,
                                                          uint64_t* table_out, uint64_t slots, int step)
{
    if (ctr->err) return;
    uint32_t q = ctr->q_in, lo, hi;
    chunk_of(q, gridDim.x, blockIdx.x, lo, hi);
    uint32_t run = blk_off[blockIdx.x];
    for (uint32_t base = lo; base < hi; base += kBlock) {
        uint32_t i = base + threadIdx.x;
        uint32_t w0 = base + (threadIdx.x & ~31u);
        uint32_t bal = (w0 < hi) ? keepw[w0 >> 5] : 0u;
        bool keep = (i < hi) && ((bal >> (threadIdx.x & 31)) & 1u);
        uint32_t tot;
        uint32_t r = block_excl_scan<kBlock>(keep ? 1u : 0u, &tot);
        if (keep) {
            uint32_t dst = run + r;
            Key<W> k = load_key<W>(keys_in, i);
            store_key<W>(keys_out, dst, k);
            c_out[dst] = c_in[i];
            if (!table_insert_unique<W>(table_out, slots, k, dst)) set_err(ctr, kErrProbe, step, 1);
        }
        run += tot;
    }
}

// ---------------------------------------------------------------- a2/a3 one level
// Insert a candidate; returns its slot if it claimed one or joined a candidate
// entry with the same key, kNone if the key is already a row (or on failure).
template <int W>
__device__ __forceinline__ uint32_t insert_candidate(const DevModel* __restrict__ M, uint64_t* table, uint64_t slots,
                                                     const Key<W>& key, uint32_t c, const uint64_t* __restrict__ keys,
                                                     uint32_t lo, Counters* ctr, int step)
{
    uint64_t h = key_hash<W>(key);
    uint64_t fp = fingerprint<W>(h);
    uint64_t mine = (fp << 32) | (uint64_t)(kCand | c);
    uint64_t pos = slot_home(h, slots);
    for (uint32_t probe = 0; probe < kMaxProbe; ++probe) {
        uint64_t* sl = table + pos * Slot<W>::kWords;
        uint64_t tag = __ldcg(sl);
        if (tag == kEmpty) {
            unsigned long long old = atomicCAS((unsigned long long*)sl, kEmpty, mine);
            if (old == kEmpty) return (uint32_t)pos;
            tag = old;
        }
        if ((tag >> 32) == fp) {
            uint32_t v = (uint32_t)tag;
            if (v & kCand) {
                // another candidate holds the slot: regenerate its key from its parent
                uint32_t c2 = v & ~kCand;
                uint32_t p2 = (uint32_t)udiv(c2, M->div_D);
                int mv2 = (int)(c2 - p2 * (uint32_t)M->D);
                Key<W> pk = load_key<W>(keys, lo + p2);
                int s2 = key_site<W>(pk, M);
                int ns2 = key_digit<W>(pk, M, s2);
                Key<W> k2;
                int cid2;
                if (apply_move<W>(M, pk, s2, ns2, mv2, k2, cid2) && key_eq<W>(k2, key)) {
                    atomicMin((unsigned long long*)sl, (unsigned long long)mine);
                    return (uint32_t)pos;
                }
            } else {
                bool eq = true;
#pragma unroll
                for (int i = 0; i < W; ++i) eq &= (__ldcg(sl + 1 + i) == key.w[i]);
                if (eq) return kNone;
            }
        }
        pos = slot_next(pos, slots);
    }
    set_err(ctr, kErrProbe, step, 2);
    return kNone;
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_level_insert(const DevModel* __restrict__ M, Counters* ctr, int f,
                                                         const uint64_t* __restrict__ keys, uint64_t* table,
                                                         uint64_t slots, uint32_t* __restrict__ cand_slot,
                                                         uint64_t cand_cap, int step)
{
    if (ctr->err) return;
    uint32_t lo = ctr->level_off[f], hi = ctr->level_off[f + 1];
    int D = M->D;
    uint64_t ncand = (uint64_t)(hi - lo) * (uint64_t)D;
    if (ncand >= (uint64_t)kCand || ncand > cand_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctr, kErrCand, step, f);
        return;
    }
    for (uint32_t p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, p);
        int s = key_site<W>(k, M);
        int ns = key_digit<W>(k, M, s);
        uint32_t cbase = (p - lo) * (uint32_t)D;
        for (int mv = 0; mv < D; ++mv) {
            Key<W> child;
            int cid;
            uint32_t r = kNone;
            if (apply_move<W>(M, k, s, ns, mv, child, cid))
                r = insert_candidate<W>(M, table, slots, child, cbase + mv, keys, lo, ctr, step);
            cand_slot[cbase + mv] = r;
        }
    }
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_level_flags(const DevModel* __restrict__ M, Counters* ctr, int f,
                                                        const uint64_t* __restrict__ table,
                                                        const uint32_t* __restrict__ cand_slot,
                                                        uint64_t* __restrict__ masks, uint32_t* __restrict__ blk_cnt)
{
    if (ctr->err) return;
    uint32_t lo0 = ctr->level_off[f], F = ctr->level_off[f + 1] - lo0, lo, hi;
    chunk_of(F, gridDim.x, blockIdx.x, lo, hi);
    int D = M->D;
    uint32_t cnt = 0;
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kBlock) {
        uint64_t m = 0;
        uint32_t cbase = i * (uint32_t)D;
        for (int mv = 0; mv < D; ++mv) {
            uint32_t sl = cand_slot[cbase + mv];
            if (sl == kNone) continue;
            uint64_t tag = table[(uint64_t)sl * Slot<W>::kWords];
            if ((uint32_t)tag == (kCand | (cbase + mv))) m |= 1ull << mv;
        }
        masks[i] = m;
        cnt += __popcll(m);
    }
    uint32_t tot;
    block_excl_scan<kBlock>(cnt, &tot);
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = tot;
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_level_scatter(const DevModel* __restrict__ M, Counters* ctr, int f,
                                                          uint64_t* keys, uint64_t* table,
                                                          const uint32_t* __restrict__ cand_slot,
                                                          const uint64_t* __restrict__ masks,
                                                          const uint32_t* __restrict__ blk_off,
                                                          const uint64_t* __restrict__ old_table, uint64_t old_slots,
                                                          const double2* __restrict__ c_old, double2* __restrict__ c_new)
{
    if (ctr->err) return;
    uint32_t lo0 = ctr->level_off[f], base_row = ctr->level_off[f + 1];
    uint32_t F = base_row - lo0, lo, hi;
    chunk_of(F, gridDim.x, blockIdx.x, lo, hi);
    int D = M->D;
    uint32_t run = blk_off[blockIdx.x];
    for (uint32_t tile = lo; tile < hi; tile += kBlock) {
        uint32_t i = tile + threadIdx.x;
        uint64_t m = (i < hi) ? masks[i] : 0ull;
        uint32_t tot;
        uint32_t r = block_excl_scan<kBlock>((uint32_t)__popcll(m), &tot);
        if (m) {
            Key<W> k = load_key<W>(keys, lo0 + i);
            int s = key_site<W>(k, M);
            int ns = key_digit<W>(k, M, s);
            uint32_t row = base_row + run + r;
            uint32_t cbase = i * (uint32_t)D;
            while (m) {
                int mv = __ffsll((long long)m) - 1;
                m &= m - 1;
                Key<W> child;
                int cid;
                apply_move<W>(M, k, s, ns, mv, child, cid);
                store_key<W>(keys, row, child);
                uint64_t* sl = table + (uint64_t)cand_slot[cbase + mv] * Slot<W>::kWords;
#pragma unroll
                for (int w = 0; w < W; ++w) sl[1 + w] = child.w[w];
                sl[0] = (sl[0] & 0xFFFFFFFF00000000ull) | (uint64_t)row;
                double2 a = make_double2(0.0, 0.0);
                if (old_table) {
                    int64_t orow = table_lookup<W>(old_table, old_slots, child);
                    if (orow >= 0) a = c_old[orow];
                }
                c_new[row] = a;
                ++row;
            }
        }
        run += tot;
    }
}

// ---------------------------------------------------------------- a5 P H P
// Row i holds the off-diagonal entries of P_m H P_m in move order (hops to
// t ascending, a_s^dag, a_s), columns = rows of the images that lie in H_eff,
// and the diagonal eps_s + sum_j omega_j n_j summed in site order.
template <int W>
__global__ void __launch_bounds__(kBlock) k_csr(const DevModel* __restrict__ M, Counters* ctr,
                                                const uint64_t* __restrict__ keys, const uint64_t* __restrict__ table,
                                                uint64_t slots, uint32_t* __restrict__ col, uint8_t* __restrict__ cidv,
                                                uint8_t* __restrict__ cnt, double* __restrict__ diag)
{
    if (ctr->err) return;
    uint32_t q = ctr->q;
    int D = M->D, P = M->P;
    unsigned long long nnz = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, i);
        uint64_t q0 = udiv(k.w[0], M->div_exc);
        int s = (int)(k.w[0] - q0 * M->div_exc.d);
        double d = M->eps[s];
        int ns = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t x = (w == 0) ? q0 : k.w[w];
            for (int j = M->word_first[w]; j < M->word_first[w + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                int nj = (int)(x - xq * M->div_radix[j].d);
                x = xq;
                d = __dadd_rn(d, __dmul_rn(M->omega[j], (double)nj));
                if (j == s) ns = nj;
            }
        }
        uint32_t e = 0;
        uint64_t rbase = (uint64_t)i * (uint64_t)P;
        for (int mv = 0; mv < D; ++mv) {
            Key<W> child;
            int cid;
            if (!apply_move<W>(M, k, s, ns, mv, child, cid)) continue;
            int64_t r = table_lookup<W>(table, slots, child);
            if (r < 0) continue;
            col[rbase + e] = (uint32_t)r;
            cidv[rbase + e] = (uint8_t)cid;
            ++e;
        }
        cnt[i] = (uint8_t)e;
        diag[i] = d;
        nnz += e;
    }
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

__device__ __forceinline__ void split_weight(double w, unsigned long long& hi, unsigned long long& lo)
{
    double x = w * 4503599627370496.0;          // 2^52, exact
    double f = floor(x);
    hi = (unsigned long long)f;
    lo = (unsigned long long)((x - f) * 4294967296.0);   // next 32 bits, truncated
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_accum(const DevModel* __restrict__ M, Counters* ctr,
                                                      const uint64_t* __restrict__ keys,
                                                      const double2* __restrict__ vec,
                                                      unsigned long long* __restrict__ part)
{
    __shared__ unsigned long long sh_hi[kObsStride], sh_lo[kObsStride];
    if (ctr->err) return;
    const int N = M->N;
    for (int t = threadIdx.x; t < 2 * N + 1; t += blockDim.x) sh_hi[t] = sh_lo[t] = 0ull;
    __syncthreads();
    const uint32_t q = ctr->q;
    unsigned long long nh = 0, nl = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        double2 v = vec[i];
        double w = v.x * v.x + v.y * v.y;
        if (w == 0.0) continue;
        unsigned long long hi, lo;
        split_weight(w, hi, lo);
        nh += hi;
        nl += lo;
        Key<W> k = load_key<W>(keys, i);
        uint64_t q0 = udiv(k.w[0], M->div_exc);
        int s = (int)(k.w[0] - q0 * M->div_exc.d);
        atomicAdd(&sh_hi[s], hi);
        atomicAdd(&sh_lo[s], lo);
#pragma unroll
        for (int wd = 0; wd < W; ++wd) {
            uint64_t x = (wd == 0) ? q0 : k.w[wd];
            for (int j = M->word_first[wd]; j < M->word_first[wd + 1] && x; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                unsigned long long nj = x - xq * M->div_radix[j].d;
                x = xq;
                if (nj) {
                    atomicAdd(&sh_hi[N + j], hi * nj);
                    atomicAdd(&sh_lo[N + j], lo * nj);
                }
            }
        }
    }
    atomicAdd(&sh_hi[2 * N], nh);
    atomicAdd(&sh_lo[2 * N], nl);
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * N + 1; t += blockDim.x) {
        part[((size_t)blockIdx.x * kObsStride + t) * 2] = sh_hi[t];
        part[((size_t)blockIdx.x * kObsStride + t) * 2 + 1] = sh_lo[t];
    }
}

// mode: 0 after a step, 1 the record of set_state, 2 after the first step
template <int W>
__global__ void __launch_bounds__(kBlock) k_obs_finish(const DevModel* __restrict__ M, Counters* ctr,
                                                       const uint64_t* __restrict__ table, uint64_t slots,
                                                       const uint64_t* __restrict__ psi0_keys,
                                                       const double2* __restrict__ psi0_amp, int64_t n0,
                                                       const double2* __restrict__ vec, double t, int mode,
                                                       const unsigned long long* __restrict__ part, int nparts,
                                                       double* __restrict__ rec)
{
    if (ctr->err) return;
    const int N = M->N;
    __shared__ double nrm;
    for (int i = threadIdx.x; i < 2 * N + 1; i += blockDim.x) {
        unsigned long long hi = 0, lo = 0;
        for (int b = 0; b < nparts; ++b) {
            hi += part[((size_t)b * kObsStride + i) * 2];
            lo += part[((size_t)b * kObsStride + i) * 2 + 1];
        }
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
        double2 a = psi0_amp[k], c = vec[r];
        acc[0] += a.x * c.x + a.y * c.y;    // conj(a) * c
        acc[1] += a.x * c.y - a.y * c.x;
    }
    __shared__ double cs[2];
    block_sum<kBlock, 2>(acc, cs);
    if (threadIdx.x == 0) {
        bool initial = mode == 1;
        if (mode == 2) ctr->kept = ctr->q;      // the first step propagates every row
        double norm = initial ? nrm : ctr->norm_r;
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
        ctr->norm_last = norm;
        ctr->nnz = 0;            // the next step's P H P build counts from zero
    }
}

// ---------------------------------------------------------------- export helpers
template <int W>
__global__ void k_decode(const DevModel* __restrict__ M, const uint64_t* __restrict__ keys, uint32_t n,
                         int32_t* __restrict__ site, int32_t* __restrict__ occ)
{
    int N = M->N;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Key<W> k = load_key<W>(keys, i);
        uint64_t q0 = udiv(k.w[0], M->div_exc);
        site[i] = (int32_t)(k.w[0] - q0 * M->div_exc.d);
        for (int w = 0; w < W; ++w) {
            uint64_t x = (w == 0) ? q0 : k.w[w];
            for (int j = M->word_first[w]; j < M->word_first[w + 1]; ++j) {
                uint64_t xq = udiv(x, M->div_radix[j]);
                occ[(uint64_t)i * N + j] = (int32_t)(x - xq * M->div_radix[j].d);
                x = xq;
            }
        }
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
static int trunc_w(const Bufs& b, int gin, int gout, double th2, int step, cudaStream_t st)
{
    k_trunc_count<<<b.G, kBlock, 0, st>>>(b.V[0], b.ctr, th2, b.keepw, b.blk_cnt);
    k_scan<<<1, 1024, 0, st>>>(b.blk_cnt, b.blk_off, b.G, b.ctr, kScanTrunc, 0, b.cap_rows, step);
    k_trunc_scatter<W><<<b.G, kBlock, 0, st>>>(b.keys[gin], b.V[0], b.ctr, b.keepw, b.blk_off, b.keys[gout],
                                               b.V[1], b.table[gout], b.table_slots, step);
    return 3;
}

template <int W>
static int level_w(const Bufs& b, int gen, int f, int rescue_gen, int step, cudaStream_t st)
{
    k_level_insert<W><<<b.grid, kBlock, 0, st>>>(b.model, b.ctr, f, b.keys[gen], b.table[gen], b.table_slots,
                                                 b.cand_slot, b.cand_cap, step);
    k_level_flags<W><<<b.G, kBlock, 0, st>>>(b.model, b.ctr, f, b.table[gen], b.cand_slot, b.masks, b.blk_cnt);
    k_scan<<<1, 1024, 0, st>>>(b.blk_cnt, b.blk_off, b.G, b.ctr, kScanLevel, f, b.cap_rows, step);
    const uint64_t* ot = rescue_gen >= 0 ? b.table[rescue_gen] : nullptr;
    k_level_scatter<W><<<b.G, kBlock, 0, st>>>(b.model, b.ctr, f, b.keys[gen], b.table[gen], b.cand_slot,
                                               b.masks, b.blk_off, ot, b.table_slots, b.V[0], b.V[1]);
    return 4;
}

template <int W>
static int csr_w(const Bufs& b, int gen, cudaStream_t st)
{
    k_csr<W><<<b.grid, kBlock, 0, st>>>(b.model, b.ctr, b.keys[gen], b.table[gen], b.table_slots, b.col, b.cid,
                                        b.cnt, b.diag);
    return 1;
}

template <int W>
static int observe_w(const Bufs& b, int gen, const double2* vec, double t, int64_t rec, int mode, cudaStream_t st)
{
    double* r = b.obs + rec * b.rec_len;
    k_obs_accum<W><<<b.grid, kBlock, 0, st>>>(b.model, b.ctr, b.keys[gen], vec, b.obs_part);
    k_obs_finish<W><<<1, kBlock, 0, st>>>(b.model, b.ctr, b.table[gen], b.table_slots, b.psi0_keys, b.psi0_amp,
                                          b.n0, vec, t, mode, b.obs_part, b.grid, r);
    return 2;
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

int launch_level(const Bufs& b, int gen, int f, int rescue_gen, int step, cudaStream_t st)
{
    PACES_DISPATCH_W(b.W, level_w<KW>(b, gen, f, rescue_gen, step, st))
}

int launch_csr(const Bufs& b, int gen, cudaStream_t st) { PACES_DISPATCH_W(b.W, csr_w<KW>(b, gen, st)) }

int launch_observe(const Bufs& b, int gen, const double2* vec, double t, int64_t rec, int mode, cudaStream_t st)
{
    PACES_DISPATCH_W(b.W, observe_w<KW>(b, gen, vec, t, rec, mode, st))
}

int launch_decode(const Bufs& b, int gen, uint32_t n, int32_t* site, int32_t* occ, cudaStream_t st)
{
    int grid = b.grid;
    PACES_DISPATCH_W(b.W, (k_decode<KW><<<grid, kBlock, 0, st>>>(b.model, b.keys[gen], n, site, occ), 1))
}

int launch_export_csr(const Bufs& b, uint32_t q, const uint64_t* off, int32_t* cols, double* vals, cudaStream_t st)
{
    k_export_csr<<<b.grid, kBlock, 0, st>>>(b.model, q, off, b.col, b.cid, b.cnt, cols, vals);
    return 1;
}

}  // namespace paces
