// kern_taylor.cu -- a6: exp(-i P H P dt) c' by the Taylor series (App. C.1):
//   phi_0 = c',  phi_n = (-i dt / n) (P H P) phi_{n-1},  r = sum_n phi_n,
// stopping at the first n >= 2 with ||phi_n||^2 <= tol^2 ||r||^2.
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
    const double2* c_in;     // phi_0 = c'
    double2* r;              // accumulator (the new state)
    double2* ta;             // term buffers
    double2* tb;
    float2* fa;              // complex64 term buffers
    float2* fb;
    double* partials;        // [2][G][4]
    double* totals;          // [2][4]
    TaylorParams p;
};

// Barrier that also reduces the per-block partials: the last block to arrive
// sums them in block order and publishes the four totals before releasing the
// others.  Every wait is bounded (kBarrierTimeoutNs).
__device__ __forceinline__ bool barrier_reduce(Counters* ctr, const double* part, double* tot, unsigned G)
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

template <int LPR>
__global__ void __launch_bounds__(kBlock) k_taylor(TaylorArgs a)
{
    __shared__ double coef[kMaxCoefs];
    __shared__ double tsh[4];
    Counters* ctr = a.ctr;
    if (ctr->err) return;
    const DevModel* M = a.M;
    for (int t = threadIdx.x; t < M->ncoef; t += blockDim.x) coef[t] = M->coef[t];
    __syncthreads();

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
    const double2* x = a.c_in;
    double2* y = a.ta;
    double E = 0.0, n0 = 0.0, r2 = 0.0;
    int nd = 0;
    bool conv = false;
    for (int n = 1; n <= nlimit; ++n) {
        const double s = a.p.dt / (double)n;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (uint32_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
            uint32_t row = rb + sub;
            bool valid = row < q;
            uint32_t c = valid ? a.cnt[row] : 0u;
            uint64_t base = (uint64_t)row * P;
            double2 yv = row_apply<LPR, double2>(a.col, a.cid, c, base, coef, x, lane);
            if (valid && lane == 0) {
                double2 xi = x[row];
                double d = a.diag[row];
                yv.x = fma(d, xi.x, yv.x);
                yv.y = fma(d, xi.y, yv.y);
                double2 phi = make_double2(s * yv.y, -s * yv.x);     // (-i s) y
                y[row] = phi;
                double2 rr = (n == 1) ? xi : a.r[row];
                rr.x += phi.x;
                rr.y += phi.y;
                a.r[row] = rr;
                acc[0] += phi.x * phi.x + phi.y * phi.y;
                acc[1] += rr.x * rr.x + rr.y * rr.y;
                if (n == 1) {
                    acc[2] += xi.x * yv.x + xi.y * yv.y;            // Re(conj(c') H c')
                    acc[3] += xi.x * xi.x + xi.y * xi.y;
                }
            }
        }
        double* part = a.partials + (size_t)(n & 1) * G * 4;
        double* tot = a.totals + (n & 1) * 4;
        block_sum<kBlock, 4>(acc, part + 4 * blockIdx.x);
        if (!barrier_reduce(ctr, part, tot, G)) return;
        if (threadIdx.x < 4) tsh[threadIdx.x] = __ldcg(tot + threadIdx.x);
        __syncthreads();
        nd = n;
        r2 = tsh[1];
        if (n == 1) {
            E = tsh[2];
            n0 = tsh[3];
        }
        if (fixed <= 0 && n >= 2 && tsh[0] <= a.p.tol2 * tsh[1]) {
            conv = true;
            break;
        }
        x = y;
        y = (y == a.ta) ? a.tb : a.ta;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->nterms = nd;
        ctr->norm_r = r2;
        ctr->norm_phi0 = n0;
        ctr->energy = E;
        if (!conv && fixed <= 0 && atomicCAS(&ctr->err, 0, (int)kErrNoConverge) == 0) {
            ctr->err_step = a.p.step;
            ctr->err_info = nd;
        }
    }
}

template <int LPR>
static int occupancy()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_taylor<LPR>, kBlock, 0);
    return nb;
}

int taylor_blocks_per_sm(int lpr, int c64)
{
    (void)c64;
    if (lpr == 1) return occupancy<1>();
    if (lpr == 4) return occupancy<4>();
    return occupancy<8>();
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
    a.c_in = b.V[1];
    a.r = b.V[0];
    a.ta = b.V[2];
    a.tb = b.V[3];
    a.fa = b.F[0];
    a.fb = b.F[1];
    a.partials = b.partials;
    a.totals = b.partials + 2 * 4 * (size_t)b.taylor_grid;
    a.p = p;
    void* args[] = {&a};
    const void* fn = p.lpr == 1 ? (const void*)k_taylor<1> : p.lpr == 4 ? (const void*)k_taylor<4>
                                                                        : (const void*)k_taylor<8>;
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(b.taylor_grid), dim3(kBlock), args, 0, st);
    return e == cudaSuccess ? 1 : -1;
}

}  // namespace paces
