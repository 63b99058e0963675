// kern_adjoint.cu -- reverse pass of one propagation step (a gradient
// extension: the paper defines the forward map only).
//
// With the subspace sequence and the number of Taylor terms of every step held
// at their forward values, one step is linear in the amplitudes:
//     c' = R c                (truncation Q and regrowth with rescue, Sec. 3:
//                              a fixed injective row map "from")
//     phi_0 = c',  phi_n = (-i dt / n) H phi_{n-1},  c_new = sum_{n <= N} phi_n
// (the truncated series of the propagator, Eq. taylor).  For a real loss L with
// cotangent gbar = dL/dRe c_new + i dL/dIm c_new the reverse recurrence is
//     mu_N = gbar,   mu_{n-1} = gbar + (i dt / n) H mu_n      (H real symmetric)
// and mu_0 is the cotangent of c'; it reaches the previous rows through
// "from".  A parameter p of H receives
//     dL/dp += Re sum_i conj(mu_n,i) (-i dt / n) (dH/dp phi_{n-1})_i
//            = (dt / n) Im sum_i conj(mu_n,i) (dH/dp phi_{n-1})_i
// for n = N .. 1, with dH/dJ and dH/dg the per-entry coefficient derivatives,
// dH/domega = diag(sum_j n_j) (a common shift of all omega_j) and
// dH/deps_s = the projector on exciton site s (Eq. holstein).
//
// All adjoint arithmetic is FP64.  Per-row contributions are summed over the
// terms of a step in a per-row accumulator (each row owned by one lane group,
// so the order is fixed), then reduced into the 3 + N parameter bins as exact
// fixed-point integers (resolution 2^-72), so the gradient does not depend on
// the order in which blocks finish.
#include "runtime.h"

namespace paces {

namespace {

constexpr int kAdjBlock = 256;

// Amplitude in the storage format (16 bytes: double-word pair or FP64) as FP64.
__device__ __forceinline__ double2 load_amp(const void* v, uint64_t i, int fmt)
{
    if (fmt == 1) return reinterpret_cast<const double2*>(v)[i];
    float4 a = reinterpret_cast<const float4*>(v)[i];
    return make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
}

__device__ __forceinline__ double load_diag(const double* d, uint64_t i, int fmt)
{
    if (fmt == 1) return d[i];
    float2 a = reinterpret_cast<const float2*>(d)[i];
    return (double)a.x + (double)a.y;
}

// Im(conj(a) b)
__device__ __forceinline__ double im_conj_mul(double2 a, double2 b) { return a.x * b.y - a.y * b.x; }

// trunc(x * 2^72) as a signed 128-bit integer, exactly, from the bits of x;
// false when |x| >= 2^50 (outside the range the bins are sized for).
__device__ __forceinline__ bool fix72(double x, __int128& out)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((u >> 52) & 0x7FFull);
    unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    out = 0;
    if (ex == 0) {
        if (m == 0) return true;
        ex = 1;
    } else {
        m |= 1ull << 52;
    }
    if (ex >= 1023 + 50) return false;           // also catches inf and NaN
    int sh = ex - 1075 + 72;                     // x = m 2^(ex - 1075)
    __int128 v;
    if (sh >= 0) v = ((__int128)m) << sh;        // sh <= 46: fits in 99 bits
    else v = (sh <= -53) ? (__int128)0 : (__int128)(m >> (-sh));
    out = (u >> 63) ? -v : v;
    return true;
}

// The three 32-bit limbs of a fixed-point value as u64 addends: limbs 0 and 1
// are non-negative, limb 2 carries the sign (two's complement, wraps).
__device__ __forceinline__ void limbs(__int128 F, unsigned long long& l0, unsigned long long& l1,
                                      unsigned long long& l2)
{
    l0 = (unsigned long long)(F & 0xFFFFFFFF);
    l1 = (unsigned long long)((F >> 32) & 0xFFFFFFFF);
    l2 = (unsigned long long)(F >> 64);
}

}  // namespace

// ---------------------------------------------------------------- cotangents
// gbar_i += 2 c_i dL/dP_{s(i)}: P_s = sum over rows with exciton on s of |c_i|^2
// (the site populations of Sec. observables), c the post-step amplitudes.
__global__ void __launch_bounds__(kAdjBlock) k_adj_obs_rows(const Counters* __restrict__ ctr,
                                                            const uint32_t* __restrict__ meta,
                                                            const void* __restrict__ vec, int fmt,
                                                            const double* __restrict__ dLdP,
                                                            double2* __restrict__ gbar)
{
    const uint32_t q = ctr->q;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x) {
        double w = dLdP[meta_s(meta[i])];
        if (w == 0.0) continue;
        double2 c = load_amp(vec, i, fmt), g = gbar[i];
        g.x += 2.0 * w * c.x;
        g.y += 2.0 * w * c.y;
        gbar[i] = g;
    }
}

// gbar_row(j) += psi0_j w for C(t) = sum_j conj(psi0_j) c(key_j): with
// dL = Re(conj(w) dC) the cotangent of c(key_j) is psi0_j w.  psi(0) keys are
// distinct, so no two threads touch one row.
template <int W>
__global__ void __launch_bounds__(kAdjBlock) k_adj_obs_psi0(const uint64_t* __restrict__ table, uint64_t slots,
                                                            const uint64_t* __restrict__ psi0_keys,
                                                            const double2* __restrict__ psi0_amp, int64_t n0,
                                                            const double2* __restrict__ w_ptr,
                                                            double2* __restrict__ gbar)
{
    const double2 w = *w_ptr;
    if (w.x == 0.0 && w.y == 0.0) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n0; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = table_lookup<W>(table, slots, load_key<W>(psi0_keys, (uint64_t)j));
        if (row < 0) continue;
        double2 a = psi0_amp[j], g = gbar[row];
        g.x += a.x * w.x - a.y * w.y;
        g.y += a.x * w.y + a.y * w.x;
        gbar[row] = g;
    }
}

// ---------------------------------------------------------------- reverse term
struct AdjTermArgs {
    const DevModel* M;
    const Counters* ctr;
    const uint32_t* col;
    const uint8_t* cid;
    const uint8_t* cnt;
    const double* diag;
    const double2* mu_in;     // mu_n
    const void* phi;          // phi_{n-1}, storage format
    const double2* gbar;
    double2* mu_out;          // mu_{n-1}
    double* acc;              // [3][cap]: J, g, and the diagonal weight Im(conj(mu) phi)
    uint64_t acc_stride;
    double s;                 // dt / n
    int first;                // first term of the step: store instead of add
    int fmt;
    int P;
};

// One reverse term.  LPR lanes share a row's P H P entries; the partial sums
// of H mu, dH/dJ phi and dH/dg phi meet in a fixed xor-shuffle tree.
template <int LPR>
__global__ void __launch_bounds__(kAdjBlock) k_adj_term(AdjTermArgs a)
{
    __shared__ double cf[kMaxCoefs], cj[kMaxCoefs], cg[kMaxCoefs];
    const DevModel* M = a.M;
    for (int t = threadIdx.x; t < M->ncoef; t += blockDim.x) {
        cf[t] = M->coef[t];
        cj[t] = M->coef_dJ[t];
        cg[t] = M->coef_dg[t];
    }
    __syncthreads();
    const uint32_t q = a.ctr->q;
    constexpr uint32_t RPW = 32 / LPR;
    const int lane = (threadIdx.x & 31) % LPR;
    const uint32_t sub = (threadIdx.x & 31) / LPR;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t P = (uint64_t)a.P;
    const int fmt = a.fmt;
    // the loop bound is uniform over the warp, so every lane reaches the shuffles
    for (uint64_t rb = warp * RPW; rb < q; rb += nwarps * RPW) {
        const uint64_t row = rb + sub;
        const bool valid = row < q;
        const int c = valid ? a.cnt[row] : 0;
        double2 y = make_double2(0.0, 0.0), yj = y, yg = y;
        for (int e = lane; e < c; e += LPR) {
            uint64_t idx = row * P + e;
            uint32_t cl = a.col[idx];
            int id = a.cid[idx];
            double2 m = a.mu_in[cl], ph = load_amp(a.phi, cl, fmt);
            double v = cf[id], vj = cj[id], vg = cg[id];
            y.x += v * m.x;
            y.y += v * m.y;
            yj.x += vj * ph.x;
            yj.y += vj * ph.y;
            yg.x += vg * ph.x;
            yg.y += vg * ph.y;
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            y.x += __shfl_xor_sync(0xffffffffu, y.x, o, LPR);
            y.y += __shfl_xor_sync(0xffffffffu, y.y, o, LPR);
            yj.x += __shfl_xor_sync(0xffffffffu, yj.x, o, LPR);
            yj.y += __shfl_xor_sync(0xffffffffu, yj.y, o, LPR);
            yg.x += __shfl_xor_sync(0xffffffffu, yg.x, o, LPR);
            yg.y += __shfl_xor_sync(0xffffffffu, yg.y, o, LPR);
        }
        if (valid && lane == 0) {
            double2 mi = a.mu_in[row], pi = load_amp(a.phi, row, fmt), gi = a.gbar[row];
            double d = load_diag(a.diag, row, fmt);
            y.x += d * mi.x;
            y.y += d * mi.y;
            a.mu_out[row] = make_double2(gi.x - a.s * y.y, gi.y + a.s * y.x);   // gbar + i s H mu
            double vJ = a.s * im_conj_mul(mi, yj), vG = a.s * im_conj_mul(mi, yg), vE = a.s * im_conj_mul(mi, pi);
            double* A = a.acc + row;
            if (a.first) {
                A[0] = vJ;
                A[a.acc_stride] = vG;
                A[2 * a.acc_stride] = vE;
            } else {
                A[0] += vJ;
                A[a.acc_stride] += vG;
                A[2 * a.acc_stride] += vE;
            }
        }
    }
}

// ---------------------------------------------------------------- bins
// Reduce the per-row accumulators of one step into the 3 + N parameter bins
// [J, g, omega, eps_0 .. eps_{N-1}], each three u64 limb sums of 2^-72 fixed
// point (bins[(p * 3) + limb]).  Integer sums: the result does not depend on
// the order of the additions.
__global__ void __launch_bounds__(kAdjBlock) k_adj_bins(const DevModel* __restrict__ M, Counters* ctr,
                                                        const uint32_t* __restrict__ meta,
                                                        const double* __restrict__ acc, uint64_t acc_stride,
                                                        unsigned long long* __restrict__ bins)
{
    __shared__ unsigned long long sh[(3 + kMaxSites) * 3];
    const int N = M->N, nb = 3 * (3 + N);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) sh[t] = 0ull;
    __syncthreads();
    const uint32_t q = ctr->q;
    const int lane = threadIdx.x & 31;
    bool bad = false;
    unsigned long long r[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t nround = ((uint64_t)q + stride - 1) / stride;
    for (uint64_t k = 0; k < nround; ++k) {
        uint64_t i = k * stride + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
        __int128 F[4] = {0, 0, 0, 0};
        int s = -1;
        if (i < q) {
            uint32_t mt = meta[i];
            double aE = acc[i + 2 * acc_stride];
            bad |= !fix72(acc[i], F[0]);
            bad |= !fix72(acc[i + acc_stride], F[1]);
            bad |= !fix72((double)meta_nph(mt) * aE, F[2]);
            bad |= !fix72(aE, F[3]);
            s = meta_s(mt);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            unsigned long long l0, l1, l2;
            limbs(F[p], l0, l1, l2);
            r[3 * p] += l0;
            r[3 * p + 1] += l1;
            r[3 * p + 2] += l2;
        }
        if (s >= 0 && F[3] != 0) {
            unsigned long long l0, l1, l2;
            limbs(F[3], l0, l1, l2);
            atomicAdd(&sh[3 * (3 + s)], l0);
            atomicAdd(&sh[3 * (3 + s) + 1], l1);
            atomicAdd(&sh[3 * (3 + s) + 2], l2);
        }
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) r[t] = warp_sum_u64(r[t]);
    if (lane == 0)
        for (int t = 0; t < 9; ++t) atomicAdd(&sh[t], r[t]);
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_err(ctr, kErrGradRange, -1, 0);
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (sh[t]) atomicAdd(&bins[t], sh[t]);
}

// ---------------------------------------------------------------- scatter
// gprev[from[i]] = mu_0[i]: the cotangent of c' moved back to the rows of the
// previous state.  "from" is injective, so the stores never collide; rows of
// the previous state with no image keep the zero the caller wrote.
__global__ void __launch_bounds__(kAdjBlock) k_adj_scatter(const Counters* __restrict__ ctr,
                                                           const uint32_t* __restrict__ from,
                                                           const double2* __restrict__ mu0,
                                                           double2* __restrict__ gprev)
{
    const uint32_t q = ctr->q;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t f = from[i];
        if (f != kNone) gprev[f] = mu0[i];
    }
}

// ---------------------------------------------------------------- launchers
int launch_adj_obs(const Bufs& b, int gen, const void* vec, const double* dLdP, const double2* wC, double2* gbar,
                   cudaStream_t st)
{
    int n = 0;
    if (dLdP) {
        k_adj_obs_rows<<<b.grid, kAdjBlock, 0, st>>>(b.ctr, b.meta[gen], vec, b.fmt, dLdP, gbar);
        ++n;
    }
    if (wC && b.n0 > 0) {
        int grid = (int)std::min<int64_t>((b.n0 + kAdjBlock - 1) / kAdjBlock, (int64_t)b.grid);
        switch (b.W) {
        case 1: k_adj_obs_psi0<1><<<grid, kAdjBlock, 0, st>>>(b.table[gen], b.table_slots, b.psi0_keys, b.psi0_amp, b.n0, wC, gbar); break;
        case 2: k_adj_obs_psi0<2><<<grid, kAdjBlock, 0, st>>>(b.table[gen], b.table_slots, b.psi0_keys, b.psi0_amp, b.n0, wC, gbar); break;
        case 3: k_adj_obs_psi0<3><<<grid, kAdjBlock, 0, st>>>(b.table[gen], b.table_slots, b.psi0_keys, b.psi0_amp, b.n0, wC, gbar); break;
        case 4: k_adj_obs_psi0<4><<<grid, kAdjBlock, 0, st>>>(b.table[gen], b.table_slots, b.psi0_keys, b.psi0_amp, b.n0, wC, gbar); break;
        default: return -1;
        }
        ++n;
    }
    return n;
}

int launch_adj_term(const Bufs& b, int lpr, const double2* mu_in, const void* phi, const double2* gbar,
                    double2* mu_out, double* acc, uint64_t acc_stride, double s, int first, cudaStream_t st)
{
    AdjTermArgs a;
    a.M = b.model;
    a.ctr = b.ctr;
    a.col = b.col;
    a.cid = b.cid;
    a.cnt = b.cnt;
    a.diag = b.diag;
    a.mu_in = mu_in;
    a.phi = phi;
    a.gbar = gbar;
    a.mu_out = mu_out;
    a.acc = acc;
    a.acc_stride = acc_stride;
    a.s = s;
    a.first = first;
    a.fmt = b.fmt;
    a.P = b.P;
    switch (lpr) {
    case 1: k_adj_term<1><<<b.grid, kAdjBlock, 0, st>>>(a); break;
    case 2: k_adj_term<2><<<b.grid, kAdjBlock, 0, st>>>(a); break;
    case 4: k_adj_term<4><<<b.grid, kAdjBlock, 0, st>>>(a); break;
    case 8: k_adj_term<8><<<b.grid, kAdjBlock, 0, st>>>(a); break;
    default: k_adj_term<16><<<b.grid, kAdjBlock, 0, st>>>(a); break;
    }
    return 1;
}

int launch_adj_bins(const Bufs& b, int gen, const double* acc, uint64_t acc_stride, unsigned long long* bins,
                    cudaStream_t st)
{
    k_adj_bins<<<b.grid, kAdjBlock, 0, st>>>(b.model, b.ctr, b.meta[gen], acc, acc_stride, bins);
    return 1;
}

int launch_adj_scatter(const Bufs& b, const uint32_t* from, const double2* mu0, double2* gprev, cudaStream_t st)
{
    if (!from) return -1;
    k_adj_scatter<<<b.grid, kAdjBlock, 0, st>>>(b.ctr, from, mu0, gprev);
    return 1;
}

}  // namespace paces
