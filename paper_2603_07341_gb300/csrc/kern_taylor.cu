// kern_taylor.cu -- a6: exp(-i P H P dt) c' by the Taylor series (App. C.1):
//   phi_0 = c',  phi_n = (-i dt / n) (P H P) phi_{n-1},  r = sum_n phi_n,
// stopping at the first n >= 2 with ||phi_n||^2 <= tol^2 ||r||^2.
//
// Three arithmetic variants share the structure below: k_taylor_f64 keeps the
// amplitudes in FP64 (the paper's complex128); k_taylor_dw keeps every
// amplitude as a double-word (FP32 pair) and accumulates each row with the
// compensated dot product (FP32 pipe, 48-bit significand); k_taylor_c64 runs
// the later terms in complex64.
//
// One cooperative launch runs every term of a step: each term is one pass of
// SpMV over the row-pitched P H P fused with the scaling, the accumulation
// r += phi_n and the FP64 norm partials; the term ends at a grid barrier whose
// last arriving block sums the partials in a fixed order and publishes the
// totals, so all blocks take the same stop decision with no host round trip.
#include "runtime.h"

namespace paces {

struct TaylorArgs {
    const DevModel* M;
    Counters* ctr;
    const uint32_t* col;
    const uint8_t* cid;
    const uint8_t* cnt;
    const double* diag;
    double* diag_h;          // FP64 variant: h times the diagonal, formed in the first term
    const uint8_t* rperm;    // FP64 variant: rows of each 256-row window by entry count
    const double2* c_in;     // phi_0 = c'
    double2* r;              // accumulator (the new state)
    double2* ta;             // term buffers
    double2* tb;
    float2* fa;              // complex64 term buffers
    float2* fb;
    double* partials;        // [2][G][4]
    double* totals;          // [2][4]
    void* terms;             // adjoint re-runs: phi_n stored at [(n - 1) * q + row]
    int term_max;
    double2* kry;            // Lanczos: s_2 .. s_{kmax+1}, kry_stride rows apart
    uint64_t kry_stride;
    TaylorParams p;
};

// Barrier that also reduces the per-block partials: the last block to arrive
// sums them in block order and publishes the four totals before releasing the
// others.  Every wait is bounded (timeout_ns, kBarrierTimeoutNs by default):
// a wait that runs out records kErrBarrier and the block returns false.
__device__ __forceinline__ bool barrier_reduce(Counters* ctr, const double* part, double* tot, unsigned G,
                                               uint64_t timeout_ns = kBarrierTimeoutNs)
{
    __shared__ int last, ok;
    __threadfence();          // publish this thread's partial before the block arrives
    __syncthreads();
    unsigned g = 0;
    if (threadIdx.x == 0) {
        ok = 1;
        g = *(volatile unsigned*)&ctr->bar_gen;
        __threadfence();
        last = (atomicAdd(&ctr->bar_count, 1u) + 1u == G);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (unsigned b = threadIdx.x; b < G; b += blockDim.x) {
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += __ldcg(part + 4 * b + k);
        }
        __shared__ double s[4];
        block_sum<kBlock, 4>(acc, s);
        if (threadIdx.x < 4) tot[threadIdx.x] = s[threadIdx.x];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(&ctr->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctr->bar_gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        uint64_t t0 = global_ns();
        while (*(volatile unsigned*)&ctr->bar_gen == g) {
            __nanosleep(20);
            if (global_ns() - t0 > timeout_ns) {
                atomicCAS(&ctr->err, 0, (int)kErrBarrier);
                ok = 0;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Self-test of the bounded wait: every block arrives at a barrier that expects
// `expect` arrivals.  With expect == gridDim.x it completes; with more, no block
// is the last to arrive, every wait runs out after timeout_ns and kErrBarrier is
// recorded, and the kernel returns with the context intact.
__global__ void __launch_bounds__(kBlock) k_barrier_selftest(Counters* ctr, double* part, double* tot,
                                                             unsigned expect, unsigned long long timeout_ns)
{
    double z[4] = {1.0, 0.0, 0.0, 0.0};
    block_sum<kBlock, 4>(z, part + 4 * blockIdx.x);
    barrier_reduce(ctr, part, tot, expect, timeout_ns);
}

// y_row = (P H P x)_row for the rows of one warp round; LPR lanes per row.
template <int LPR, typename XT>
__device__ __forceinline__ double2 row_apply(const uint32_t* __restrict__ col, const uint8_t* __restrict__ cid,
                                             uint32_t c, uint64_t base, const double* coef,
                                             const XT* __restrict__ x, int lane)
{
    double yr = 0.0, yi = 0.0;
    if constexpr (LPR == 1) {
        for (uint32_t e = 0; e < c; e += 4) {
            uint4 cc = *reinterpret_cast<const uint4*>(col + base + e);
            uint32_t ii = *reinterpret_cast<const uint32_t*>(cid + base + e);
            uint32_t cs[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (e + k < c) {
                    double a = coef[(ii >> (8 * k)) & 0xFFu];
                    auto xv = x[cs[k]];
                    yr = fma(a, (double)xv.x, yr);
                    yi = fma(a, (double)xv.y, yi);
                }
            }
        }
    } else {
        for (uint32_t e = lane; e < c; e += LPR) {
            double a = coef[cid[base + e]];
            auto xv = x[col[base + e]];
            yr = fma(a, (double)xv.x, yr);
            yi = fma(a, (double)xv.y, yi);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            yr += __shfl_xor_sync(0xffffffffu, yr, o, LPR);
            yi += __shfl_xor_sync(0xffffffffu, yi, o, LPR);
        }
    }
    return make_double2(yr, yi);
}

// Number of Taylor series a step runs as (App. C.1's scaling alternative):
// s = ceil(rho dt / xmax), rho = the row bound of P H P that the build of the
// step's Hamiltonian left in the counters (in units of 2^-20); 1 when xmax <= 0;
// 0 when more than kMaxSub series would be needed.
__device__ __forceinline__ int series_count(const Counters* ctr, const TaylorParams& p)
{
    if (p.xmax <= 0.0) return 1;
    double rho = (double)__ldcg(&ctr->hbound) * (1.0 / 1048576.0);
    double ns = ceil(rho * p.dt / p.xmax);
    if (ns > (double)kMaxSub) return 0;
    return ns < 1.0 ? 1 : (int)ns;
}

// Rows of every 256-row window ordered by their entry count, largest first
// (stable: equal counts keep row order): rperm[w + k] = offset in window w of
// its k-th row.  The FP64 propagator gives each warp 32 consecutive ranks, so
// the rows of a warp have (nearly) equal counts and few warps issue FP64
// products for entries that only some of their rows have.  A window is one
// block's rows of one round, so the rows' own data stay within 256 rows (2048-
// row windows were measured: 1.5x the DRAM traffic, no fewer idle FP64 lanes).
// Deterministic, so that replays repeat the reduction order bit for bit.
__global__ void __launch_bounds__(kBlock) k_row_order(const Counters* __restrict__ ctr, const uint8_t* __restrict__ cnt,
                                                      int pmax, uint8_t* __restrict__ rperm)
{
    __shared__ uint32_t off[kMaxMoves + 1][kBlock / 32];
    if (ctr->err) return;
    const uint32_t q = ctr->q;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t wb = blockIdx.x * kBlock; wb < q; wb += gridDim.x * kBlock) {
        const uint32_t row = wb + threadIdx.x;
        const int c = row < q ? (int)cnt[row] : -1;
        for (int k = 0; k <= pmax; ++k) {
            const unsigned bal = __ballot_sync(0xffffffffu, c == k);
            if (lane == 0) off[k][warp] = (uint32_t)__popc(bal);
        }
        __syncthreads();
        if (threadIdx.x == 0) {            // exclusive offsets: counts descending, then warps in order
            uint32_t acc = 0;
            for (int k = pmax; k >= 0; --k)
                for (int w = 0; w < kBlock / 32; ++w) {
                    const uint32_t v = off[k][w];
                    off[k][w] = acc;
                    acc += v;
                }
        }
        __syncthreads();
        const unsigned peers = __match_any_sync(0xffffffffu, c);       // rows past q match only each other
        if (c >= 0) rperm[wb + off[c][warp] + __popc(peers & ((1u << lane) - 1u))] = (uint8_t)threadIdx.x;
        __syncthreads();
    }
}

// FP64 amplitudes.  The FP64 pipe of this part retires about two operations
// per SM per clock, so the kernel spends FP64 operations on the amplitudes
// only.  With B = h P H P (h = dt / series), the series is evaluated through
// the unscaled powers psi_n = B psi_{n-1}, psi_0 = v (the series' input), and
// r = sum_n (-i)^n / n! psi_n: B's off-diagonal entries live in a shared table
// and its diagonal h d is formed once per step, so a row of c off-diagonal
// entries costs 2c + 4 FP64 operations per term (the products, the diagonal,
// and r += (-i)^n psi_n / n! as two FMAs).  ||psi_n|| <= (rho h)^n ||v|| stays
// far inside the FP64 range for the series lengths substepping allows.
//
// Rows are taken in 256-row windows, one per block, in the order k_row_order
// leaves (one lane per row), so that a warp's 32 rows have nearly equal entry
// counts; models with more entries per row use LPR lanes per row in row order.
//
// The stop test compares ||phi_n||^2 = ||psi_n||^2 / n!^2, summed in FP32 from
// the leading 20 bits of every component of psi_n (scaled by 2^-L, 2^L <= n!,
// in the integer exponent field), with tol^2 ||v||^2 (||v|| in FP64 from the
// first term): the partial sum r_n differs from v in norm by about
// ||phi_{n+1}||, far below the test's resolution when the test is near to
// passing.  A term more or less changes r by at most tol ||v||.
//
// A step of several series copies the output of one series, held in r, into
// a term buffer as the input of the next, so that r is updated in place while
// that input is gathered.  Adjoint re-runs store, in order, the terms
// phi_1.. of the first series, then for each later series its input and its
// terms (16 bytes per row each).
template <int LPR>
__global__ void __launch_bounds__(kBlock, LPR == 1 ? 4 : 1) k_taylor_f64(TaylorArgs a)
{
    __shared__ double coef[kMaxCoefs];
    __shared__ double tsh[4];
    Counters* ctr = a.ctr;
    if (ctr->err) return;
    const DevModel* M = a.M;
    const int ncoef = M->ncoef;
    const uint32_t q = ctr->q;
    const uint64_t P = (uint64_t)M->P;
    const unsigned G = gridDim.x;
    constexpr uint32_t RPW = 32 / LPR;                       // rows per warp round
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (G * blockDim.x) >> 5;
    const int lane = (threadIdx.x & 31) % LPR;
    const uint32_t sub = (threadIdx.x & 31) / LPR;

    const int fixed = a.p.fixed_terms;
    const int nlimit = fixed > 0 ? fixed : a.p.nmax;
    const int nsub = series_count(ctr, a.p);
    if (nsub < 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctr, kErrNoConverge, a.p.step, -1);
        return;
    }
    const double h = a.p.dt / (double)nsub;
    for (int t = threadIdx.x; t < ncoef; t += blockDim.x) coef[t] = h * M->coef[t];
    __syncthreads();
    double2* store = reinterpret_cast<double2*>(a.terms);
    double E = 0.0, n0 = 0.0;
    int total = 0, slot = 0, bar = 0;
    bool conv = true;
    // r is updated at even n with both terms of the pair (n - 1, n); a series
    // that stops at an odd n leaves r += i pend_s psi_n (pend_y) to be added
    const double2* pend_y = nullptr;
    const double2* pend_b = nullptr;                // r, or v when the series stopped at n = 1
    double pend_s = 0.0;
    for (int j = 0; j < nsub && conv; ++j) {
        const double2* x = a.c_in;
        double2* y = a.ta;
        if (j > 0) {
            for (uint32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < q; row += G * blockDim.x) {
                double2 v = pend_y ? pend_b[row] : a.r[row];
                if (pend_y) {
                    const double2 pv = pend_y[row];
                    v.x = fma(-pend_s, pv.y, v.x);
                    v.y = fma(pend_s, pv.x, v.y);
                }
                a.ta[row] = v;
                if (store && slot < a.term_max) store[(size_t)slot * q + row] = v;
            }
            ++slot;
            double z[4] = {0.0, 0.0, 0.0, 0.0};
            double* part = a.partials + (size_t)(bar & 1) * G * 4;
            double* tot = a.totals + (bar & 1) * 4;
            ++bar;
            block_sum<kBlock, 4>(z, part + 4 * blockIdx.x);
            if (!barrier_reduce(ctr, part, tot, G)) return;
            x = a.ta;
            y = a.tb;
        }
        pend_y = nullptr;
        const double2* vin = x;                     // the series' input v
        const double2* last = nullptr;              // buffer holding psi_nd
        double nin = 0.0, cn = 1.0;                 // cn = 1 / n!
        int nd = 0;
        bool cj = fixed > 0;
        for (int n = 1; n <= nlimit; ++n) {
            const double cprev = cn;                 // 1 / (n - 1)!
            cn = cn / (double)n;
            const int L = -ilogb(cn);                // 2^(L-1) < n! <= 2^L
            const double corr = ldexp(cn, L);        // 2^L / n!, in [1, 2)
            // (-i)^n = s_re + i s_im with one of them +-1, the other 0
            const int ph = n & 3;
            const double sr = ph == 0 ? cn : (ph == 2 ? -cn : 0.0);
            const double si = ph == 1 ? -cn : (ph == 3 ? cn : 0.0);
            // n even: (-i)^(n-1) = i sip
            const double sip = ph == 2 ? -cprev : cprev;
            const bool first = (j == 0 && n == 1);
            float phi2 = 0.f;
            double acc_e = 0.0, acc_n = 0.0;
            const bool odd = (n & 1) != 0;
            // the row's own amplitude, B's diagonal and the accumulator
            auto load_row = [&](uint32_t row, double2& xi, double& d, double2& rr) {
                xi = x[row];
                d = first ? a.diag[row] : a.diag_h[row];
                if (!odd) rr = (n == 2) ? vin[row] : a.r[row];
            };
            auto finish_row = [&](uint32_t row, double2 yv, double2 xi, double d, double2 rr) {
                if (first) {
                    d = h * d;
                    a.diag_h[row] = d;
                }
                yv.x = fma(d, xi.x, yv.x);
                yv.y = fma(d, xi.y, yv.y);                // psi_n = B x
                y[row] = yv;
                // n even: r += i sip psi_{n-1} + sr psi_n (x holds psi_{n-1});
                // r is neither read nor written at odd n
                if (!odd) {
                    rr.x = fma(sr, yv.x, fma(-sip, xi.y, rr.x));
                    rr.y = fma(sr, yv.y, fma(sip, xi.x, rr.y));
                    a.r[row] = rr;
                }
                if (store && slot < a.term_max)
                    store[(size_t)slot * q + row] = make_double2(sr * yv.x - si * yv.y, sr * yv.y + si * yv.x);
                float p0 = mag_scaled_f32(yv.x, L), p1 = mag_scaled_f32(yv.y, L);
                phi2 = __fmaf_rn(p0, p0, __fmaf_rn(p1, p1, phi2));
                if (n == 1) {
                    acc_e = fma(xi.x, yv.x, fma(xi.y, yv.y, acc_e));     // Re(conj(v) h H v)
                    acc_n = fma(xi.x, xi.x, fma(xi.y, xi.y, acc_n));
                }
            };
            if constexpr (LPR == 1) {
                // one 256-row window per block and round, rows by entry count;
                // every load of a row (its entries, their amplitudes, its own
                // amplitude, diagonal and accumulator) is issued before its
                // first FP64 operation
                for (uint32_t wb = blockIdx.x * kBlock; wb < q; wb += G * kBlock) {
                    const uint32_t sl = wb + threadIdx.x;
                    const uint32_t row = sl < q ? wb + a.rperm[sl] : q;
                    const bool valid = row < q;
                    const uint32_t c = valid ? a.cnt[row] : 0u;
                    const uint64_t base = (uint64_t)row * P;
                    uint4 cc = make_uint4(0, 0, 0, 0);
                    uint32_t ii = 0;
                    if (c > 0) {
                        cc = *reinterpret_cast<const uint4*>(a.col + base);
                        ii = *reinterpret_cast<const uint32_t*>(a.cid + base);
                    }
                    const uint32_t cs[4] = {cc.x, cc.y, cc.z, cc.w};
                    double2 xv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) xv[k] = c > (uint32_t)k ? x[cs[k]] : make_double2(0.0, 0.0);
                    double2 xi = make_double2(0.0, 0.0), rr = xi;
                    double d = 0.0;
                    if (valid) load_row(row, xi, d, rr);
                    double yr = 0.0, yi = 0.0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (__any_sync(0xffffffffu, c > (uint32_t)k)) {
                            const double av = c > (uint32_t)k ? coef[(ii >> (8 * k)) & 0xFFu] : 0.0;
                            yr = fma(av, xv[k].x, yr);
                            yi = fma(av, xv[k].y, yi);
                        }
                    }
                    for (uint32_t e = 4; e < c; e += 4) {      // pitches above 4 (P <= 8)
                        const uint4 c2 = *reinterpret_cast<const uint4*>(a.col + base + e);
                        const uint32_t i2 = *reinterpret_cast<const uint32_t*>(a.cid + base + e);
                        const uint32_t cs2[4] = {c2.x, c2.y, c2.z, c2.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (e + k < c) {
                                const double av = coef[(i2 >> (8 * k)) & 0xFFu];
                                const double2 xw = x[cs2[k]];
                                yr = fma(av, xw.x, yr);
                                yi = fma(av, xw.y, yi);
                            }
                        }
                    }
                    if (valid) finish_row(row, make_double2(yr, yi), xi, d, rr);
                }
            } else {
                for (uint32_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
                    uint32_t row = rb + sub;
                    bool valid = row < q;
                    uint32_t c = valid ? a.cnt[row] : 0u;
                    uint64_t base = (uint64_t)row * P;
                    double2 yv = row_apply<LPR, double2>(a.col, a.cid, c, base, coef, x, lane);
                    if (valid && lane == 0) {
                        double2 xi, rr;
                        double d;
                        load_row(row, xi, d, rr);
                        finish_row(row, yv, xi, d, rr);
                    }
                }
            }
            ++slot;
            double acc[4] = {(double)phi2, acc_e, acc_n, 0.0};
            double* part = a.partials + (size_t)(bar & 1) * G * 4;
            double* tot = a.totals + (bar & 1) * 4;
            ++bar;
            block_sum<kBlock, 4>(acc, part + 4 * blockIdx.x);
            if (!barrier_reduce(ctr, part, tot, G)) return;
            if (threadIdx.x < 4) tsh[threadIdx.x] = __ldcg(tot + threadIdx.x);
            __syncthreads();
            nd = n;
            last = y;
            if (n == 1) {
                nin = tsh[2];
                if (j == 0) {
                    E = tsh[1] / h;
                    n0 = tsh[2];
                }
            }
            // sum f^2 = ||phi_n||^2 2^64 / corr^2
            if (fixed <= 0 && n >= 2 && tsh[0] * corr * corr <= a.p.tol2 * nin * 18446744073709551616.0) {
                cj = true;
                break;
            }
            x = y;
            y = (y == a.ta) ? a.tb : a.ta;
        }
        total += nd;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr->sub_terms[j] = nd;
        conv = cj;
        if (nd & 1) {                               // (-i)^nd / nd! = i pend_s
            pend_y = last;
            pend_b = nd == 1 ? vin : a.r;
            pend_s = (nd & 3) == 1 ? -cn : cn;
        }
    }
    if (pend_y && conv) {                           // the last series stopped at an odd n
        for (uint32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < q; row += G * blockDim.x) {
            double2 v = pend_b[row];
            const double2 pv = pend_y[row];
            v.x = fma(-pend_s, pv.y, v.x);
            v.y = fma(pend_s, pv.x, v.y);
            a.r[row] = v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nterms = total;
        ctr->nsub = nsub;
        ctr->norm_r = 0.0;
        ctr->norm_phi0 = n0;
        ctr->energy = E;
        if (!conv && atomicCAS(&ctr->err, 0, (int)kErrNoConverge) == 0) {
            ctr->err_step = a.p.step;
            ctr->err_info = total;
        }
    }
}

// ---------------------------------------------------------------- double-word variant
struct Red8 {
    float phi2, r2;
    dwf e, n0;
};

__device__ __forceinline__ Red8 red8_add(const Red8& x, const Red8& y)
{
    return {__fadd_rn(x.phi2, y.phi2), __fadd_rn(x.r2, y.r2), dw_add(x.e, y.e), dw_add(x.n0, y.n0)};
}

__device__ __forceinline__ Red8 red8_shfl_xor(const Red8& v, int o)
{
    Red8 r;
    r.phi2 = __shfl_xor_sync(0xffffffffu, v.phi2, o);
    r.r2 = __shfl_xor_sync(0xffffffffu, v.r2, o);
    r.e.hi = __shfl_xor_sync(0xffffffffu, v.e.hi, o);
    r.e.lo = __shfl_xor_sync(0xffffffffu, v.e.lo, o);
    r.n0.hi = __shfl_xor_sync(0xffffffffu, v.n0.hi, o);
    r.n0.lo = __shfl_xor_sync(0xffffffffu, v.n0.lo, o);
    return r;
}

// Fixed-order block reduction; the result is valid in thread 0.
__device__ __forceinline__ Red8 red8_block(Red8 v)
{
    __shared__ Red8 ws[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) v = red8_add(v, red8_shfl_xor(v, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kBlock / 32; ++w) v = red8_add(v, ws[w]);
    __syncthreads();
    return v;
}

__device__ __forceinline__ void red8_store(float* p, const Red8& v)
{
    p[0] = v.phi2; p[1] = v.r2; p[2] = v.e.hi; p[3] = v.e.lo; p[4] = v.n0.hi; p[5] = v.n0.lo;
}

__device__ __forceinline__ Red8 red8_load(const float* p)
{
    return {__ldcg(p), __ldcg(p + 1), {__ldcg(p + 2), __ldcg(p + 3)}, {__ldcg(p + 4), __ldcg(p + 5)}};
}

// Grid barrier whose last arriving block reduces the per-block partials (8
// floats each) in block order and publishes the totals.  Bounded waits.
__device__ __forceinline__ bool barrier_reduce8(Counters* ctr, const float* part, float* tot, unsigned G)
{
    __shared__ int last, ok;
    __threadfence();
    __syncthreads();
    unsigned g = 0;
    if (threadIdx.x == 0) {
        ok = 1;
        g = *(volatile unsigned*)&ctr->bar_gen;
        __threadfence();
        last = (atomicAdd(&ctr->bar_count, 1u) + 1u == G);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        Red8 acc{0.f, 0.f, {0.f, 0.f}, {0.f, 0.f}};
        for (unsigned b = threadIdx.x; b < G; b += blockDim.x) acc = red8_add(acc, red8_load(part + 8 * b));
        acc = red8_block(acc);
        if (threadIdx.x == 0) red8_store(tot, acc);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(&ctr->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctr->bar_gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        uint64_t t0 = global_ns();
        while (*(volatile unsigned*)&ctr->bar_gen == g) {
            __nanosleep(20);
            if (global_ns() - t0 > kBarrierTimeoutNs) {
                atomicCAS(&ctr->err, 0, (int)kErrBarrier);
                ok = 0;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Accumulate the off-diagonal entries of one row into Dot2 accumulators.
template <int LPR>
__device__ __forceinline__ void row_apply_dw(const uint32_t* __restrict__ col, const uint8_t* __restrict__ cid,
                                             uint32_t c, uint64_t base, const dwf* coef,
                                             const float4* __restrict__ x, int lane, Dot2& re, Dot2& im)
{
    if constexpr (LPR == 1) {
        for (uint32_t e = 0; e < c; e += 4) {
            uint4 cc = *reinterpret_cast<const uint4*>(col + base + e);
            uint32_t ii = *reinterpret_cast<const uint32_t*>(cid + base + e);
            uint32_t cs[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (e + k < c) {
                    dwf a = coef[(ii >> (8 * k)) & 0xFFu];
                    float4 xv = x[cs[k]];
                    dot2_mac(re, a, xv.x, xv.y);
                    dot2_mac(im, a, xv.z, xv.w);
                }
            }
        }
    } else {
        for (uint32_t e = lane; e < c; e += LPR) {
            dwf a = coef[cid[base + e]];
            float4 xv = x[col[base + e]];
            dot2_mac(re, a, xv.x, xv.y);
            dot2_mac(im, a, xv.z, xv.w);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            float s2 = __shfl_xor_sync(0xffffffffu, re.s, o, LPR), c2 = __shfl_xor_sync(0xffffffffu, re.c, o, LPR);
            dwf t = two_sum(re.s, s2);
            re.s = t.hi;
            re.c = __fadd_rn(__fadd_rn(re.c, c2), t.lo);
            s2 = __shfl_xor_sync(0xffffffffu, im.s, o, LPR);
            c2 = __shfl_xor_sync(0xffffffffu, im.c, o, LPR);
            t = two_sum(im.s, s2);
            im.s = t.hi;
            im.c = __fadd_rn(__fadd_rn(im.c, c2), t.lo);
        }
    }
}

template <int LPR>
__global__ void __launch_bounds__(kBlock) k_taylor_dw(TaylorArgs a)
{
    __shared__ dwf coef[kMaxCoefs];
    __shared__ float tsh[8];
    Counters* ctr = a.ctr;
    if (ctr->err) return;
    const DevModel* M = a.M;
    const int ncoef = M->ncoef;
    const uint32_t q = ctr->q;
    const uint64_t P = (uint64_t)M->P;
    const unsigned G = gridDim.x;
    constexpr uint32_t RPW = 32 / LPR;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (G * blockDim.x) >> 5;
    const int lane = (threadIdx.x & 31) % LPR;
    const uint32_t sub = (threadIdx.x & 31) / LPR;
    float4* TA = reinterpret_cast<float4*>(a.ta);
    float4* TB = reinterpret_cast<float4*>(a.tb);
    float4* R = reinterpret_cast<float4*>(a.r);
    float4* store = reinterpret_cast<float4*>(a.terms);
    const float2* DG = reinterpret_cast<const float2*>(a.diag);
    const float kScale = 4294967296.0f;       // 2^32: keeps the coarse norms in FP32 range

    const int fixed = a.p.fixed_terms;
    const int nlimit = fixed > 0 ? fixed : a.p.nmax;
    const float tol2 = (float)a.p.tol2;
    const int nsub = series_count(ctr, a.p);
    if (nsub < 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctr, kErrNoConverge, a.p.step, -1);
        return;
    }
    const double h = a.p.dt / (double)nsub;
    dwf E{0.f, 0.f}, N0{0.f, 0.f};
    int total = 0, slot = 0, bar = 0;
    bool conv = true;
    for (int j = 0; j < nsub && conv; ++j) {
        const float4* X = reinterpret_cast<const float4*>(a.c_in);
        float4* Y = TA;
        if (j > 0) {            // input of this series = output of the previous one, copied out of r
            for (uint32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < q; row += G * blockDim.x) {
                float4 v = R[row];
                TA[row] = v;
                if (store && slot < a.term_max) store[(size_t)slot * q + row] = v;
            }
            ++slot;
            float* part = reinterpret_cast<float*>(a.partials) + (size_t)(bar & 1) * G * 8;
            float* tot = reinterpret_cast<float*>(a.totals) + (bar & 1) * 8;
            ++bar;
            Red8 z = red8_block(Red8{0.f, 0.f, {0.f, 0.f}, {0.f, 0.f}});
            if (threadIdx.x == 0) red8_store(part + 8 * blockIdx.x, z);
            if (!barrier_reduce8(ctr, part, tot, G)) return;
            X = TA;
            Y = TB;
        }
        int nd = 0;
        bool cj = fixed > 0;
        for (int n = 1; n <= nlimit; ++n) {
            const double s = h / (double)n;
            const dwf sdw = dw_from_double(s);
            __syncthreads();
            for (int t = threadIdx.x; t < ncoef; t += blockDim.x) coef[t] = dw_from_double(s * M->coef[t]);
            __syncthreads();
            Red8 acc{0.f, 0.f, {0.f, 0.f}, {0.f, 0.f}};
            for (uint32_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
                uint32_t row = rb + sub;
                bool valid = row < q;
                uint32_t c = valid ? a.cnt[row] : 0u;
                uint64_t base = (uint64_t)row * P;
                Dot2 re{0.f, 0.f}, im{0.f, 0.f};
                row_apply_dw<LPR>(a.col, a.cid, c, base, coef, X, lane, re, im);
                if (valid && lane == 0) {
                    float4 xi = X[row];
                    float2 d = DG[row];
                    dwf ds = dw_mul(dwf{d.x, d.y}, sdw);
                    dot2_mac(re, ds, xi.x, xi.y);
                    dot2_mac(im, ds, xi.z, xi.w);
                    dwf yre = dot2_result(re), yim = dot2_result(im);      // y = s H x
                    float4 phi = make_float4(yim.hi, yim.lo, -yre.hi, -yre.lo);   // phi = -i y
                    Y[row] = phi;
                    if (store && slot < a.term_max) store[(size_t)slot * q + row] = phi;
                    float4 rr = (n == 1) ? xi : R[row];
                    dwf r_re = dw_add(dwf{rr.x, rr.y}, dwf{phi.x, phi.y});
                    dwf r_im = dw_add(dwf{rr.z, rr.w}, dwf{phi.z, phi.w});
                    R[row] = make_float4(r_re.hi, r_re.lo, r_im.hi, r_im.lo);
                    float p0 = phi.x * kScale, p1 = phi.z * kScale, q0 = r_re.hi * kScale, q1 = r_im.hi * kScale;
                    acc.phi2 = __fmaf_rn(p0, p0, __fmaf_rn(p1, p1, acc.phi2));
                    acc.r2 = __fmaf_rn(q0, q0, __fmaf_rn(q1, q1, acc.r2));
                    if (n == 1 && j == 0) {
                        acc.e = dw_add(acc.e, dw_add(dw_mul(dwf{xi.x, xi.y}, yre), dw_mul(dwf{xi.z, xi.w}, yim)));
                        acc.n0 = dw_add(acc.n0, dw_norm2(xi));
                    }
                }
            }
            ++slot;
            float* part = reinterpret_cast<float*>(a.partials) + (size_t)(bar & 1) * G * 8;
            float* tot = reinterpret_cast<float*>(a.totals) + (bar & 1) * 8;
            ++bar;
            acc = red8_block(acc);
            if (threadIdx.x == 0) red8_store(part + 8 * blockIdx.x, acc);
            if (!barrier_reduce8(ctr, part, tot, G)) return;
            if (threadIdx.x < 6) tsh[threadIdx.x] = __ldcg(tot + threadIdx.x);
            __syncthreads();
            nd = n;
            if (n == 1 && j == 0) {
                E = dwf{tsh[2], tsh[3]};
                N0 = dwf{tsh[4], tsh[5]};
            }
            if (fixed <= 0 && n >= 2 && tsh[0] <= tol2 * tsh[1]) {
                cj = true;
                break;
            }
            X = Y;
            Y = (Y == TA) ? TB : TA;
        }
        total += nd;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr->sub_terms[j] = nd;
        conv = cj;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nterms = total;
        ctr->nsub = nsub;
        ctr->norm_phi0 = (double)N0.hi + (double)N0.lo;
        ctr->energy = ((double)E.hi + (double)E.lo) / h;
        ctr->norm_r = 0.0;
        if (!conv && atomicCAS(&ctr->err, 0, (int)kErrNoConverge) == 0) {
            ctr->err_step = a.p.step;
            ctr->err_info = total;
        }
    }
}

// ---------------------------------------------------------------- complex64 terms
// PACES_C64_SPMV: the leading terms run as in k_taylor_dw; once a term is small
// against the state, the later terms of the series run in plain complex64 (FP32
// products and sums, coefficients rounded to FP32), each phi_n stored as float2
// and added into the double-word accumulator r with an error-free sum.  The
// switch is taken from the norms the stop test already reduces: when term m
// ends with ||phi_m||^2 <= kC64Tau2 ||r||^2, terms from max(m + 2, kDwTerms + 1)
// on run in complex64 (term m has written its result in double-word, the input
// format of a double-word term, so term m + 1 stays double-word and writes its
// own result rounded to float2 for the first complex64 term).  Every block
// reads the same reduced norms, so the whole grid switches at the same term.
// An FP32 term's rounding is about 2^-24 (c + 2) of its own norm, so with
// tau = 2^-16 what the complex64 terms add to a step's error stays near 2^-38
// of ||v|| (||phi_{m+2}|| is at most tau ||v|| (rho h)^2 / ((m + 1)(m + 2))),
// and a 2048-step run stays far inside a 1e-6 observable tolerance.  With the
// first terms of a series in double-word and the rest in FP32, the series
// costs less the faster its terms decay.
constexpr int kDwTerms = 2;                  // terms that always run double-word
constexpr float kC64Tau2 = 2.3283064365386963e-10f;   // tau^2 = 2^-32

// double-word + float (Joldes et al., DWPlusFP, Alg. 4)
__device__ __forceinline__ dwf dw_add_f(dwf x, float y)
{
    dwf s = two_sum(x.hi, y);
    float v = __fadd_rn(x.lo, s.lo);
    return fast_two_sum(s.hi, v);
}

template <int LPR>
__device__ __forceinline__ float2 row_apply_f32(const uint32_t* __restrict__ col, const uint8_t* __restrict__ cid,
                                                uint32_t c, uint64_t base, const float* coef,
                                                const float2* __restrict__ x, int lane)
{
    float yr = 0.f, yi = 0.f;
    if constexpr (LPR == 1) {
        for (uint32_t e = 0; e < c; e += 4) {
            uint4 cc = *reinterpret_cast<const uint4*>(col + base + e);
            uint32_t ii = *reinterpret_cast<const uint32_t*>(cid + base + e);
            uint32_t cs[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (e + k < c) {
                    float a = coef[(ii >> (8 * k)) & 0xFFu];
                    float2 xv = x[cs[k]];
                    yr = __fmaf_rn(a, xv.x, yr);
                    yi = __fmaf_rn(a, xv.y, yi);
                }
            }
        }
    } else {
        for (uint32_t e = lane; e < c; e += LPR) {
            float a = coef[cid[base + e]];
            float2 xv = x[col[base + e]];
            yr = __fmaf_rn(a, xv.x, yr);
            yi = __fmaf_rn(a, xv.y, yi);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            yr += __shfl_xor_sync(0xffffffffu, yr, o, LPR);
            yi += __shfl_xor_sync(0xffffffffu, yi, o, LPR);
        }
    }
    return make_float2(yr, yi);
}

template <int LPR>
__global__ void __launch_bounds__(kBlock) k_taylor_c64(TaylorArgs a)
{
    __shared__ dwf coef[kMaxCoefs];
    __shared__ float coef32[kMaxCoefs];
    __shared__ float tsh[8];
    Counters* ctr = a.ctr;
    if (ctr->err) return;
    const DevModel* M = a.M;
    const int ncoef = M->ncoef;
    const uint32_t q = ctr->q;
    const uint64_t P = (uint64_t)M->P;
    const unsigned G = gridDim.x;
    constexpr uint32_t RPW = 32 / LPR;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (G * blockDim.x) >> 5;
    const int lane = (threadIdx.x & 31) % LPR;
    const uint32_t sub = (threadIdx.x & 31) / LPR;
    float4* Y = reinterpret_cast<float4*>(a.ta);
    float4* Y2 = reinterpret_cast<float4*>(a.tb);   // input copy of series after the first
    // double-word terms alternate between the two buffers: odd terms write Y,
    // even terms Y2 (after the first series, term 2 overwrites the series
    // input copy, which only term 1 reads)
    float4* R = reinterpret_cast<float4*>(a.r);
    float2* F[2] = {a.fa, a.fb};
    const float2* DG = reinterpret_cast<const float2*>(a.diag);
    const float kScale = 4294967296.0f;

    const int fixed = a.p.fixed_terms;
    const int nlimit = fixed > 0 ? fixed : a.p.nmax;
    const float tol2 = (float)a.p.tol2;
    const int nsub = series_count(ctr, a.p);
    if (nsub < 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctr, kErrNoConverge, a.p.step, -1);
        return;
    }
    const double h = a.p.dt / (double)nsub;
    dwf E{0.f, 0.f}, N0{0.f, 0.f};
    int total = 0, bar = 0;
    bool conv = true;
    for (int j = 0; j < nsub && conv; ++j) {
        const float4* X = reinterpret_cast<const float4*>(a.c_in);
        if (j > 0) {
            for (uint32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < q; row += G * blockDim.x) Y2[row] = R[row];
            float* part = reinterpret_cast<float*>(a.partials) + (size_t)(bar & 1) * G * 8;
            float* tot = reinterpret_cast<float*>(a.totals) + (bar & 1) * 8;
            ++bar;
            Red8 z = red8_block(Red8{0.f, 0.f, {0.f, 0.f}, {0.f, 0.f}});
            if (threadIdx.x == 0) red8_store(part + 8 * blockIdx.x, z);
            if (!barrier_reduce8(ctr, part, tot, G)) return;
            X = Y2;
        }
        int nd = 0;
        bool cj = fixed > 0;
        int c64_from = nlimit + 2;                  // first complex64 term (none yet)
        for (int n = 1; n <= nlimit; ++n) {
            const double s = h / (double)n;
            const dwf sdw = dw_from_double(s);
            const float s32 = (float)s;
            const bool dw_term = n < c64_from;
            const bool dw_next = n + 1 < c64_from;  // the format term n + 1 reads
            __syncthreads();
            for (int t = threadIdx.x; t < ncoef; t += blockDim.x) {
                coef[t] = dw_from_double(s * M->coef[t]);
                coef32[t] = (float)(s * M->coef[t]);
            }
            __syncthreads();
            const float4* Xd = (n == 1) ? X : ((n & 1) ? Y2 : Y);             // double-word input
            const float2* Xf = F[(n + 1) & 1];                               // complex64 input
            float2* Yf = F[n & 1];                                           // complex64 output
            Red8 acc{0.f, 0.f, {0.f, 0.f}, {0.f, 0.f}};
            for (uint32_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
                uint32_t row = rb + sub;
                bool valid = row < q;
                uint32_t c = valid ? a.cnt[row] : 0u;
                uint64_t base = (uint64_t)row * P;
                float4 phi;
                if (dw_term) {
                    Dot2 re{0.f, 0.f}, im{0.f, 0.f};
                    row_apply_dw<LPR>(a.col, a.cid, c, base, coef, Xd, lane, re, im);
                    if (!(valid && lane == 0)) continue;
                    float4 xi = Xd[row];
                    float2 d = DG[row];
                    dwf ds = dw_mul(dwf{d.x, d.y}, sdw);
                    dot2_mac(re, ds, xi.x, xi.y);
                    dot2_mac(im, ds, xi.z, xi.w);
                    dwf yre = dot2_result(re), yim = dot2_result(im);
                    phi = make_float4(yim.hi, yim.lo, -yre.hi, -yre.lo);
                    if (dw_next) ((n & 1) ? Y : Y2)[row] = phi;
                    else Yf[row] = make_float2(phi.x + phi.y, phi.z + phi.w);   // next input, rounded
                    if (n == 1 && j == 0) {
                        acc.e = dw_add(acc.e, dw_add(dw_mul(dwf{xi.x, xi.y}, yre), dw_mul(dwf{xi.z, xi.w}, yim)));
                        acc.n0 = dw_add(acc.n0, dw_norm2(xi));
                    }
                } else {
                    float2 yv = row_apply_f32<LPR>(a.col, a.cid, c, base, coef32, Xf, lane);
                    if (!(valid && lane == 0)) continue;
                    float2 xi = Xf[row];
                    float2 d = DG[row];
                    float ds = __fmul_rn(d.x + d.y, s32);
                    yv.x = __fmaf_rn(ds, xi.x, yv.x);
                    yv.y = __fmaf_rn(ds, xi.y, yv.y);
                    Yf[row] = make_float2(yv.y, -yv.x);
                    phi = make_float4(yv.y, 0.f, -yv.x, 0.f);
                }
                float4 rr = (n == 1) ? X[row] : R[row];
                dwf r_re = dw_term ? dw_add(dwf{rr.x, rr.y}, dwf{phi.x, phi.y}) : dw_add_f(dwf{rr.x, rr.y}, phi.x);
                dwf r_im = dw_term ? dw_add(dwf{rr.z, rr.w}, dwf{phi.z, phi.w}) : dw_add_f(dwf{rr.z, rr.w}, phi.z);
                R[row] = make_float4(r_re.hi, r_re.lo, r_im.hi, r_im.lo);
                float p0 = phi.x * kScale, p1 = phi.z * kScale, q0 = r_re.hi * kScale, q1 = r_im.hi * kScale;
                acc.phi2 = __fmaf_rn(p0, p0, __fmaf_rn(p1, p1, acc.phi2));
                acc.r2 = __fmaf_rn(q0, q0, __fmaf_rn(q1, q1, acc.r2));
            }
            float* part = reinterpret_cast<float*>(a.partials) + (size_t)(bar & 1) * G * 8;
            float* tot = reinterpret_cast<float*>(a.totals) + (bar & 1) * 8;
            ++bar;
            acc = red8_block(acc);
            if (threadIdx.x == 0) red8_store(part + 8 * blockIdx.x, acc);
            if (!barrier_reduce8(ctr, part, tot, G)) return;
            if (threadIdx.x < 6) tsh[threadIdx.x] = __ldcg(tot + threadIdx.x);
            __syncthreads();
            nd = n;
            if (n == 1 && j == 0) {
                E = dwf{tsh[2], tsh[3]};
                N0 = dwf{tsh[4], tsh[5]};
            }
            if (fixed <= 0 && n >= 2 && tsh[0] <= tol2 * tsh[1]) {
                cj = true;
                break;
            }
            if (c64_from > nlimit && tsh[0] <= kC64Tau2 * tsh[1]) c64_from = max(n + 2, kDwTerms + 1);
        }
        total += nd;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr->sub_terms[j] = nd;
        conv = cj;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nterms = total;
        ctr->nsub = nsub;
        ctr->norm_phi0 = (double)N0.hi + (double)N0.lo;
        ctr->energy = ((double)E.hi + (double)E.lo) / h;
        ctr->norm_r = 0.0;
        if (!conv && atomicCAS(&ctr->err, 0, (int)kErrNoConverge) == 0) {
            ctr->err_step = a.p.step;
            ctr->err_info = total;
        }
    }
}

// ---------------------------------------------------------------- Lanczos (App. C.3)
// y = exp(-i h T) e_1 for the j x j symmetric tridiagonal T (diagonal al[0..j-1],
// off-diagonal be[0..j-2]), one lane per component (j <= 32): the Taylor series
// u_n = (-i h / n) T u_{n-1}, y = sum_n u_n, until ||u_n||^2 <= 1e-34 ||y||^2.
// Warp sums by an xor butterfly give every lane the same bits, so every lane
// (and every block, from the same al, be) takes the same decisions.
__device__ __forceinline__ double warp_allsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ void tri_exp_e1(const double* al, const double* be, int j, double h, int lane, double& yr, double& yi)
{
    const double a = lane < j ? al[lane] : 0.0;
    const double bl = (lane >= 1 && lane < j) ? be[lane - 1] : 0.0;
    const double bu = (lane + 1 < j) ? be[lane] : 0.0;
    double ur = lane == 0 ? 1.0 : 0.0, ui = 0.0;
    yr = ur;
    yi = 0.0;
    for (int n = 1; n <= 400; ++n) {
        const double upr = __shfl_up_sync(0xffffffffu, ur, 1), upi = __shfl_up_sync(0xffffffffu, ui, 1);
        const double dnr = __shfl_down_sync(0xffffffffu, ur, 1), dni = __shfl_down_sync(0xffffffffu, ui, 1);
        const double vr = fma(a, ur, fma(bl, upr, bu * dnr));
        const double vi = fma(a, ui, fma(bl, upi, bu * dni));
        const double f = h / (double)n;
        ur = f * vi;                       // (-i f) (vr + i vi)
        ui = -f * vr;
        yr += ur;
        yi += ui;
        const double t2 = warp_allsum(fma(ur, ur, ui * ui)), y2 = warp_allsum(fma(yr, yr, yi * yi));
        if (t2 <= 1e-34 * y2) break;
    }
}

// exp(-i P H P dt) c' by the Lanczos decomposition of App. C.3,
// exp(-i h H) v ~ beta_0 V_n exp(-i h T_n) e_1, as the same s = ceil(rho dt /
// xmax) series of h = dt / s as the Taylor propagator.  The basis is kept
// unnormalised, s_1 = v and s_{j+1} = beta_j v_{j+1}, with v_k = sigma_k s_k,
// sigma_k = 1 / ||s_k||: per Krylov vector, pass A writes t = H s_j into the
// slot of s_{j+1} (SpMV with the table of H's entries, unscaled) and sums
// Re<s_j|t>, so alpha_j = sigma_j^2 Re<s_j|t>; pass B turns t in place into
// s_{j+1} = sigma_j t - alpha_j sigma_j s_j - beta_{j-1} sigma_{j-1} s_{j-1}
// and sums its norm, beta_j.  Each pass ends at the reducing grid barrier.
// Then every block computes y = exp(-i h T_j) e_1 (one warp) and stops at the
// first j with h beta_j |y_j| <= tol (the residual estimate); past kmax
// vectors the step does not converge.  The series' result
// r = ||v|| sum_k y_k sigma_k s_k is one more streaming pass.  FP64 throughout;
// one Krylov vector costs two passes and the basis kmax vectors of storage,
// against one pass and no storage per Taylor term.
template <int LPR>
__global__ void __launch_bounds__(kBlock) k_lanczos_f64(TaylorArgs a)
{
    __shared__ double coef[kMaxCoefs];
    __shared__ double al[kMaxKrylov], be[kMaxKrylov + 1], sg[kMaxKrylov + 2];
    __shared__ double yre[32], yim[32];
    __shared__ double tsh[4];
    __shared__ int sstop;
    Counters* ctr = a.ctr;
    if (ctr->err) return;
    const DevModel* M = a.M;
    const uint32_t q = ctr->q;
    const uint64_t P = (uint64_t)M->P;
    const unsigned G = gridDim.x;
    constexpr uint32_t RPW = 32 / LPR;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (G * blockDim.x) >> 5;
    const int lane = (threadIdx.x & 31) % LPR;
    const uint32_t sub = (threadIdx.x & 31) / LPR;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = G * blockDim.x;
    const int K = a.p.kmax;
    const double tol = sqrt(a.p.tol2);

    const int nsub = series_count(ctr, a.p);
    if (nsub < 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctr, kErrNoConverge, a.p.step, -1);
        return;
    }
    const double h = a.p.dt / (double)nsub;
    for (int t = threadIdx.x; t < M->ncoef; t += blockDim.x) coef[t] = M->coef[t];
    __syncthreads();
    int bar = 0;
    auto reduce = [&](double (&acc)[4]) -> bool {
        double* part = a.partials + (size_t)(bar & 1) * G * 4;
        double* tot = a.totals + (bar & 1) * 4;
        ++bar;
        block_sum<kBlock, 4>(acc, part + 4 * blockIdx.x);
        if (!barrier_reduce(ctr, part, tot, G)) return false;
        if (threadIdx.x < 4) tsh[threadIdx.x] = __ldcg(tot + threadIdx.x);
        __syncthreads();
        return true;
    };
    double E = 0.0, n0 = 0.0;
    int total = 0;
    bool conv = true;
    for (int js = 0; js < nsub && conv; ++js) {
        const double2* s1 = js == 0 ? a.c_in : a.r;
        auto S = [&](int k) -> const double2* { return k == 1 ? s1 : a.kry + (uint64_t)(k - 2) * a.kry_stride; };
        double b0 = 0.0;
        int n = 0;
        bool done = false;
        for (int j = 1; j <= K; ++j) {
            const double2* sj = S(j);
            double2* out = a.kry + (uint64_t)(j - 1) * a.kry_stride;
            // pass A: t = H s_j
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (uint32_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
                const uint32_t row = rb + sub;
                const bool valid = row < q;
                const uint32_t c = valid ? a.cnt[row] : 0u;
                double2 yv = row_apply<LPR, double2>(a.col, a.cid, c, (uint64_t)row * P, coef, sj, lane);
                if (valid && lane == 0) {
                    const double2 xi = sj[row];
                    const double d = a.diag[row];
                    yv.x = fma(d, xi.x, yv.x);
                    yv.y = fma(d, xi.y, yv.y);
                    out[row] = yv;
                    acc[0] = fma(xi.x, yv.x, fma(xi.y, yv.y, acc[0]));
                    if (j == 1) acc[1] = fma(xi.x, xi.x, fma(xi.y, xi.y, acc[1]));
                }
            }
            if (!reduce(acc)) return;
            if (j == 1) {
                b0 = sqrt(tsh[1]);
                if (js == 0) {
                    E = tsh[0];
                    n0 = tsh[1];
                }
                if (b0 == 0.0) {            // exp(..) 0 = 0
                    done = true;
                    n = 0;
                    break;
                }
                if (threadIdx.x == 0) sg[1] = 1.0 / b0;
                __syncthreads();
            }
            if (threadIdx.x == 0) al[j - 1] = sg[j] * sg[j] * tsh[0];
            __syncthreads();
            // pass B: s_{j+1} = sigma_j t - alpha_j sigma_j s_j - beta_{j-1} sigma_{j-1} s_{j-1}
            const double cs = sg[j], ca = -al[j - 1] * sg[j];
            const double cb = j > 1 ? -be[j - 1] * sg[j - 1] : 0.0;
            const double2* sm = j > 1 ? S(j - 1) : sj;
            double acc2[4] = {0.0, 0.0, 0.0, 0.0};
            for (uint32_t row = tid; row < q; row += nthr) {
                const double2 t = out[row], x = sj[row], xm = sm[row];
                double2 w;
                w.x = fma(cs, t.x, fma(ca, x.x, cb * xm.x));
                w.y = fma(cs, t.y, fma(ca, x.y, cb * xm.y));
                out[row] = w;
                acc2[0] = fma(w.x, w.x, fma(w.y, w.y, acc2[0]));
            }
            if (!reduce(acc2)) return;
            if (threadIdx.x == 0) be[j] = sqrt(tsh[0]);
            __syncthreads();
            if (threadIdx.x < 32) {
                double yr, yi;
                tri_exp_e1(al, be + 1, j, h, threadIdx.x, yr, yi);
                yre[threadIdx.x] = yr;
                yim[threadIdx.x] = yi;
                const double lr = __shfl_sync(0xffffffffu, yr, j - 1), li = __shfl_sync(0xffffffffu, yi, j - 1);
                if (threadIdx.x == 0) {
                    sstop = h * be[j] * sqrt(fma(lr, lr, li * li)) <= tol;
                    sg[j + 1] = 1.0 / be[j];
                }
            }
            __syncthreads();
            n = j;
            if (sstop) {
                done = true;
                break;
            }
        }
        total += n;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr->sub_terms[js] = n;
        if (!done) {
            conv = false;
            break;
        }
        // r = ||v|| sum_k y_k sigma_k s_k (in place over s_1 when s_1 = r)
        for (uint32_t row = tid; row < q; row += nthr) {
            double rr = 0.0, ri = 0.0;
            for (int k = 1; k <= n; ++k) {
                const double2 x = S(k)[row];
                const double f = b0 * sg[k];
                const double cr = f * yre[k - 1], ci = f * yim[k - 1];
                rr = fma(cr, x.x, fma(-ci, x.y, rr));
                ri = fma(cr, x.y, fma(ci, x.x, ri));
            }
            a.r[row] = make_double2(rr, ri);
        }
        if (js + 1 < nsub) {                // the next series gathers r
            double z[4] = {0.0, 0.0, 0.0, 0.0};
            if (!reduce(z)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nterms = total;
        ctr->nsub = nsub;
        ctr->norm_r = 0.0;
        ctr->norm_phi0 = n0;
        ctr->energy = E;
        if (!conv && atomicCAS(&ctr->err, 0, (int)kErrNoConverge) == 0) {
            ctr->err_step = a.p.step;
            ctr->err_info = total;
        }
    }
}

// Co-resident blocks per SM of the propagator variant that the precision
// selects (PACES_C128, PACES_DW or PACES_C64_SPMV).
template <int LPR>
static int occupancy(int precision)
{
    int n = 0;
    const void* fn = precision == kPrecLanczos ? (const void*)k_lanczos_f64<LPR>
                   : precision == PACES_C128 ? (const void*)k_taylor_f64<LPR>
                   : precision == PACES_C64_SPMV ? (const void*)k_taylor_c64<LPR> : (const void*)k_taylor_dw<LPR>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kBlock, 0);
    return n;
}

int taylor_blocks_per_sm(int lpr, int precision)
{
    if (lpr == 1) return occupancy<1>(precision);
    if (lpr == 4) return occupancy<4>(precision);
    return occupancy<8>(precision);
}

int launch_taylor(const Bufs& b, const TaylorParams& p, cudaStream_t st)
{
    TaylorArgs a;
    a.M = b.model;
    a.ctr = b.ctr;
    a.col = b.col;
    a.cid = b.cid;
    a.cnt = b.cnt;
    a.diag = b.diag;
    a.diag_h = b.diag_h;
    a.rperm = b.rperm;
    a.c_in = b.V[1];
    a.r = b.V[0];
    a.ta = b.V[2];
    a.tb = b.V[3];
    a.fa = b.F[0];
    a.fb = b.F[1];
    a.partials = b.partials;
    a.totals = b.partials + 2 * 4 * (size_t)b.taylor_grid;
    a.terms = b.terms;
    a.term_max = b.term_max;
    a.kry = b.kry;
    a.kry_stride = b.cap_rows;
    a.p = p;
    void* args[] = {&a};
    const void* fn;
    if (p.lanczos)
        fn = p.lpr == 1 ? (const void*)k_lanczos_f64<1> : p.lpr == 4 ? (const void*)k_lanczos_f64<4>
                                                                     : (const void*)k_lanczos_f64<8>;
    else if (p.fmt == 1)
        fn = p.lpr == 1 ? (const void*)k_taylor_f64<1> : p.lpr == 4 ? (const void*)k_taylor_f64<4>
                                                                    : (const void*)k_taylor_f64<8>;
    else if (p.c64)
        fn = p.lpr == 1 ? (const void*)k_taylor_c64<1> : p.lpr == 4 ? (const void*)k_taylor_c64<4>
                                                                    : (const void*)k_taylor_c64<8>;
    else
        fn = p.lpr == 1 ? (const void*)k_taylor_dw<1> : p.lpr == 4 ? (const void*)k_taylor_dw<4>
                                                                   : (const void*)k_taylor_dw<8>;
    // cooperative launch (all blocks co-resident for the grid barrier); the
    // launch-attribute form is also recorded by stream capture
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.taylor_grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (p.fmt == 1 && p.lpr == 1 && !p.lanczos) {   // rows of every window by entry count
        k_row_order<<<b.grid, kBlock, 0, st>>>(b.ctr, b.cnt, b.P, b.rperm);
        ++n;
    }
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    return e == cudaSuccess ? n + 1 : -1;
}

int launch_barrier_selftest(Counters* ctr, double* part, int grid, unsigned expect, unsigned long long timeout_ns,
                            cudaStream_t st)
{
    double* tot = part + 4 * (size_t)grid;
    void* args[] = {&ctr, &part, &tot, &expect, &timeout_ns};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)k_barrier_selftest, args) == cudaSuccess ? 1 : -1;
}

// ---------------------------------------------------------------- FP64 rate probe
// The FP64 FMA rate this GPU sustains, for the propagator's roofline: every
// thread runs kChains independent FMA chains a <- a m + c for `iters`
// iterations (with m = 1/2 and c = 1/4 every chain settles at 1/2, so the
// values stay finite and normal).  A store that only a chain ending at a value
// it cannot reach would take keeps the work live; g_fp64_sink is a valid
// device variable, so even that store stays in bounds.
__device__ double g_fp64_sink;

__global__ void __launch_bounds__(kBlock) k_fp64_rate(int iters, double m, double c)
{
    constexpr int kChains = 8;
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (double)((threadIdx.x + i) & 7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
    }
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) sum += a[i];
    if (sum == -1.0) g_fp64_sink = sum;
}

// Launches the probe on `grid` blocks of kBlock threads and returns the FMAs
// it issues (kChains per thread and iteration), or -1 on a launch error.
double launch_fp64_rate(int grid, int iters, cudaStream_t st)
{
    k_fp64_rate<<<grid, kBlock, 0, st>>>(iters, 0.5, 0.25);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return 8.0 * (double)grid * kBlock * (double)iters;
}

int fp64_rate_blocks_per_sm()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fp64_rate, kBlock, 0);
    return n;
}

}  // namespace paces
