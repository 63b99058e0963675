// common.cuh -- device-side building blocks of the paces hot path (sm_103a).
//
// Basis keys (App. A, mixed radix): a state (s, n_0..n_{N-1}) is stored as W
// 64-bit words; word 0 holds the exciton digit s lowest, then sites in order;
// no digit straddles a word.  Moves of H are word additions:
//   hop s -> t      : word0 += t - s
//   a_j^dag / a_j   : word[w_j] +/- stride_j           (Eq. holstein terms)
// Digits are read with division by invariant integers (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig. 4.1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace paces {

constexpr int kMaxSites = 128;
constexpr int kMaxWords = 4;
constexpr int kMaxMoves = 64;
constexpr int kMaxCoefs = 256;
constexpr int kMaxLevels = 256;
constexpr int kMaxCap = 255;          // phonon cap K_j per site
constexpr uint32_t kCand = 0x80000000u;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kMaxProbe = 1u << 16;
constexpr int kMaxSub = 1024;         // Taylor series per time step (substeps)
constexpr int kMaxKrylov = 32;        // Lanczos vectors per series (one warp lane each)

// device error codes (Counters::err)
enum DevErr : int {
    kErrNone = 0,
    kErrRows = 1,        // H_eff outgrew the row capacity
    kErrProbe = 2,       // hash probe sequence exceeded kMaxProbe (table overloaded)
    kErrCand = 3,        // candidate index space exhausted
    kErrNoConverge = 4,  // Taylor series not converged in nmax terms
    kErrBarrier = 5,     // a grid barrier waited past its time limit
    kErrGradRange = 6,   // an adjoint row contribution left the fixed-point range
};

// ---------------------------------------------------------------- division
struct UDiv {          // q = floor(n / d) for all 64-bit n
    uint64_t d, m;
    uint32_t sh1, sh2;
};

__host__ __device__ inline uint64_t udiv(uint64_t n, const UDiv& v)
{
#ifdef __CUDA_ARCH__
    uint64_t t1 = __umul64hi(v.m, n);
#else
    uint64_t t1 = (uint64_t)(((unsigned __int128)v.m * n) >> 64);
#endif
    return (t1 + ((n - t1) >> v.sh1)) >> v.sh2;
}

// ---------------------------------------------------------------- double-word arithmetic
// A double-word number is an unevaluated sum hi + lo of two FP32 values with
// |lo| <= ulp(hi) / 2: a 48-bit significand carried on the FP32 pipe.  The
// building blocks are the classical error-free transformations (TwoSum of
// Knuth, FastTwoSum of Dekker, TwoProd through an FMA) and the double-word
// algorithms analysed by Joldes, Muller and Popescu, "Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic", ACM TOMS 44(2),
// 2017: AccurateDWPlusDW (their Alg. 6, relative error <= 3u^2 + 13u^3),
// DWTimesDW3 (Alg. 12, <= 4u^2) and DWTimesFP3 (Alg. 7, <= 2u^2), u = 2^-24.
// Sums of products use the compensated dot product Dot2 of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005.
// Every operation is an explicitly rounded intrinsic so that the compiler can
// neither contract nor reorder it.
struct dwf {
    float hi, lo;
};

__host__ __device__ inline dwf dw_from_double(double v)
{
    float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ dwf fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float z = __fsub_rn(s, a);
    return {s, __fsub_rn(b, z)};
}

__device__ __forceinline__ dwf two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float ap = __fsub_rn(s, b);
    float bp = __fsub_rn(s, ap);
    float da = __fsub_rn(a, ap);
    float db = __fsub_rn(b, bp);
    return {s, __fadd_rn(da, db)};
}

__device__ __forceinline__ dwf two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dwf dw_add(dwf x, dwf y)
{
    dwf s = two_sum(x.hi, y.hi);
    dwf t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    dwf v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ dwf dw_mul(dwf x, dwf y)
{
    float ch = __fmul_rn(x.hi, y.hi);
    float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(cl1, cl2);
    return fast_two_sum(ch, cl3);
}

__device__ __forceinline__ dwf dw_mul_f(dwf x, float y)
{
    float ch = __fmul_rn(x.hi, y);
    float cl1 = __fmaf_rn(x.hi, y, -ch);
    float cl3 = __fmaf_rn(x.lo, y, cl1);
    return fast_two_sum(ch, cl3);
}

__device__ __forceinline__ dwf dw_neg(dwf x) { return {-x.hi, -x.lo}; }

// Dot2 accumulator: s carries the rounded running sum, c the sum of the
// rounding errors of every product and addition.
struct Dot2 {
    float s, c;
};

__device__ __forceinline__ void dot2_mac(Dot2& a, dwf coef, float xh, float xl)
{
    dwf p = two_prod(coef.hi, xh);
    float e = __fmaf_rn(coef.hi, xl, p.lo);
    e = __fmaf_rn(coef.lo, xh, e);
    dwf t = two_sum(a.s, p.hi);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ dwf dot2_result(const Dot2& a) { return two_sum(a.s, a.c); }

// |c|^2 of a double-word complex (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ dwf dw_norm2(float4 v)
{
    dwf re{v.x, v.y}, im{v.z, v.w};
    return dw_add(dw_mul(re, re), dw_mul(im, im));
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// trunc(f * 2^84) as a signed 128-bit integer, exactly, from the bits of f
// (finite f with |f| < 2^40).
__device__ __forceinline__ __int128 fix84(float f)
{
    unsigned u = __float_as_uint(f);
    int ex = (int)((u >> 23) & 0xFFu);
    unsigned m = u & 0x7FFFFFu;
    if (ex == 0) {
        if (m == 0) return 0;
        ex = 1;
    } else {
        m |= 0x800000u;
    }
    int sh = ex - 150 + 84;                      // f = m 2^(ex - 150)
    __int128 v;
    if (sh >= 0) v = ((__int128)m) << sh;
    else v = (sh <= -24) ? (__int128)0 : (__int128)(m >> (-sh));
    return (u >> 31) ? -v : v;
}

// ---------------------------------------------------------------- model
// Everything the kernels need to know about one model, resident in device
// memory (read through the read-only path).
struct DevModel {
    int N, W, D, P;            // sites, key words, max moves, row pitch of P H P
    int pow2;
    int nlad;                  // ladder table entries
    UDiv div_exc;              // word0 / exciton radix (N, or the next power of two)
    UDiv div_D;                // candidate index / D
    int word_first[kMaxWords + 1];   // sites of word w: [word_first[w], word_first[w+1])
    int site_word[kMaxSites];
    uint64_t stride[kMaxSites];
    UDiv div_stride[kMaxSites];
    UDiv div_radix[kMaxSites];
    int cap[kMaxSites];
    int gnz[kMaxSites];        // g_s != 0
    double eps[kMaxSites];
    double omega[kMaxSites];
    dwf eps_dw[kMaxSites];
    dwf omega_dw[kMaxSites];
    int uniform_omega;         // all omega_j equal (diagonal = eps_s + omega sum_j n_j)
    int uniform_radix;         // all site radices equal (one divisor decodes every digit)
    // one-word keys with a uniform radix R and at most 16 sites, when
    // R^8 (R - 1) < 2^32: the phonon digits split into two 32-bit halves of at
    // most 8 digits (q0 = h R^8 + l), each decoded with 32-bit multiplies by
    // r_magic = ceil(2^32 / R), exact for every half below 2^32 / (R - 1)
    int r8_ok;
    uint32_t r_magic;
    UDiv div_r8;
    int batch;                 // realisations R of an ensemble (1: one model)
    int batch_word;            // realisation digit: word, place value, radix
    UDiv div_batch_stride;
    UDiv div_batch_radix;
    const double* eps_b64;     // ensembles: eps[r * N + s] (FP64), device memory
    const dwf* eps_bdw;        // ensembles: eps[r * N + s] (double-word)
    int fmt;                   // amplitude storage: 0 double-word, 1 FP64
    int ncoef_pad;
    int adj_off[kMaxSites + 1];  // hops of site s: adj[adj_off[s] .. adj_off[s+1]) ascending t
    int lad_off[kMaxSites + 1];  // ladder cids of site s: lad_cid[lad_off[s] + k] = cid(g_s sqrt(k+1))
    uint8_t adj[kMaxSites * (kMaxMoves - 2)];
    uint8_t adj_cid[kMaxSites * (kMaxMoves - 2)];
    double coef[kMaxCoefs];
    // bound on ||P H P||: every term |x| rounded up to a multiple of 2^-20 and
    // held as an integer (up20), so that row sums are exact and order-free
    unsigned long long hb_coef[kMaxCoefs];   // up20(|coef|)
    unsigned long long hb_eps[kMaxSites];    // up20(|eps_s|) (single model)
    unsigned long long hb_omega[kMaxSites];  // up20(|omega_j|)
    unsigned long long hb_hop[kMaxSites];    // sum over the hops t of s of up20(|J_ts|)
    double coef_dJ[kMaxCoefs];
    double coef_dg[kMaxCoefs];
    int ncoef;
    uint8_t lad_cid[kMaxSites * kMaxCap];
};

// Per-handle counters shared by the kernels of a step (device memory).
struct Counters {
    uint32_t q;                      // rows of the current H_eff
    uint32_t q_in;                   // rows of the state that entered the step
    uint32_t kept;                   // |M|
    uint32_t nlevels;                // levels recorded in level_off (count - 1)
    uint32_t level_off[kMaxLevels + 2];
    unsigned long long nnz;          // off-diagonal entries of P H P
    int err, err_step, err_info, pad0;
    unsigned bar_count, bar_gen;
    int nterms, pad1;
    int nsub, pad2;                  // Taylor series of the last step (substeps)
    unsigned long long hbound;       // largest row bound of P H P in 2^-20 units (a5)
    double norm_r, norm_phi0, energy, norm_last;
    double time;                     // t of the last record
    long long rec_index;             // next observables record
    int sub_terms[kMaxSub];          // terms of each series of the last step
};

// Record the first device error (code, step, detail); later ones are dropped.
__device__ __forceinline__ void set_err(Counters* ctr, int code, int step, int info)
{
    if (atomicCAS(&ctr->err, 0, code) == 0) {
        ctr->err_step = step;
        ctr->err_info = info;
    }
}

// ---------------------------------------------------------------- keys
template <int W>
struct Key {
    uint64_t w[W];
};

template <int W>
__device__ __forceinline__ Key<W> load_key(const uint64_t* __restrict__ keys, uint64_t row)
{
    Key<W> k;
    const uint64_t* p = keys + row * W;
    if constexpr (W == 2) {
        ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
        k.w[0] = v.x;
        k.w[1] = v.y;
    } else if constexpr (W == 4) {
        ulonglong2 a = reinterpret_cast<const ulonglong2*>(p)[0];
        ulonglong2 b = reinterpret_cast<const ulonglong2*>(p)[1];
        k.w[0] = a.x; k.w[1] = a.y; k.w[2] = b.x; k.w[3] = b.y;
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) k.w[i] = p[i];
    }
    return k;
}

template <int W>
__device__ __forceinline__ void store_key(uint64_t* __restrict__ keys, uint64_t row, const Key<W>& k)
{
    uint64_t* p = keys + row * W;
#pragma unroll
    for (int i = 0; i < W; ++i) p[i] = k.w[i];
}

template <int W>
__device__ __forceinline__ bool key_eq(const Key<W>& a, const Key<W>& b)
{
    bool e = true;
#pragma unroll
    for (int i = 0; i < W; ++i) e &= (a.w[i] == b.w[i]);
    return e;
}

// exciton site s of a key
template <int W>
__device__ __forceinline__ int key_site(const Key<W>& k, const DevModel* M)
{
    uint64_t q = udiv(k.w[0], M->div_exc);
    return (int)(k.w[0] - q * M->div_exc.d);
}

// phonon number at site j
template <int W>
__device__ __forceinline__ int key_digit(const Key<W>& k, const DevModel* M, int j)
{
    uint64_t x = k.w[M->site_word[j]];
    uint64_t q = udiv(x, M->div_stride[j]);
    uint64_t q2 = udiv(q, M->div_radix[j]);
    return (int)(q - q2 * M->div_radix[j].d);
}

// Realisation index of a key (0 for a single model).
template <int W>
__device__ __forceinline__ int key_real(const Key<W>& k, const DevModel* M)
{
    if (M->batch <= 1) return 0;
    uint64_t q = udiv(k.w[M->batch_word], M->div_batch_stride);
    uint64_t q2 = udiv(q, M->div_batch_radix);
    return (int)(q - q2 * M->div_batch_radix.d);
}

// Per-row descriptor kept beside the key so that moves need no digit
// decoding: exciton site s (bits 0-7), phonons at s (8-15), total phonon
// number (16-31).
__host__ __device__ inline uint32_t meta_pack(int s, int ns, int nph)
{
    return (uint32_t)s | ((uint32_t)ns << 8) | ((uint32_t)nph << 16);
}
__device__ __forceinline__ int meta_s(uint32_t m) { return (int)(m & 0xFFu); }
__device__ __forceinline__ int meta_ns(uint32_t m) { return (int)((m >> 8) & 0xFFu); }
__device__ __forceinline__ int meta_nph(uint32_t m) { return (int)(m >> 16); }

// MurmurHash3 64-bit finaliser (Appleby), applied word by word.
__device__ __forceinline__ uint64_t fmix64(uint64_t h)
{
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

template <int W>
__device__ __forceinline__ uint64_t key_hash(const Key<W>& k)
{
    uint64_t h = fmix64(k.w[0] + 0x9E3779B97F4A7C15ull);
#pragma unroll
    for (int i = 1; i < W; ++i) h = fmix64(h ^ k.w[i]);
    return h;
}

// Move mv of a state with exciton site s and n_s phonons there:
//   mv < deg(s): hop to the mv-th neighbour (ascending site index)
//   mv == deg(s): a_s^dag (valid if g_s != 0 and n_s < K_s)
//   mv == deg(s)+1: a_s    (valid if g_s != 0 and n_s > 0)
// Returns false for an invalid move; on success writes the child and its
// coefficient id.
template <int W>
__device__ __forceinline__ bool apply_move(const DevModel* M, const Key<W>& k,
                                           int s, int ns, int mv, Key<W>& child, int& cid)
{
    int a0 = M->adj_off[s], deg = M->adj_off[s + 1] - a0;
    child = k;
    if (mv < deg) {
        int t = M->adj[a0 + mv];
        child.w[0] = k.w[0] + (uint64_t)t - (uint64_t)s;
        cid = M->adj_cid[a0 + mv];
        return true;
    }
    if (!M->gnz[s]) return false;
    const int w = W == 1 ? 0 : M->site_word[s];
    if (mv == deg) {
        if (ns >= M->cap[s]) return false;
        child.w[w] = k.w[w] + M->stride[s];
        cid = M->lad_cid[M->lad_off[s] + ns];
        return true;
    }
    if (mv == deg + 1) {
        if (ns <= 0) return false;
        child.w[w] = k.w[w] - M->stride[s];
        cid = M->lad_cid[M->lad_off[s] + ns - 1];
        return true;
    }
    return false;
}

// Descriptor of the state reached from (key, m) by move mv (a valid move).
template <int W>
__device__ __forceinline__ uint32_t child_meta(const DevModel* M, const Key<W>& k, uint32_t m, int mv)
{
    int s = meta_s(m), ns = meta_ns(m), nph = meta_nph(m);
    int a0 = M->adj_off[s], deg = M->adj_off[s + 1] - a0;
    if (mv < deg) {
        int t = M->adj[a0 + mv];
        return meta_pack(t, key_digit<W>(k, M, t), nph);
    }
    if (mv == deg) return meta_pack(s, ns + 1, nph + 1);
    return meta_pack(s, ns - 1, nph - 1);
}

// ---------------------------------------------------------------- hash table
// Open addressing with linear probing.  Slot = tag word (fingerprint << 32 |
// value) followed by the W key words, padded to a multiple of 16 bytes.
// value = row index, or kCand | candidate index while a level is being built.
template <int W>
struct Slot {
    static constexpr int kWords = (W == 1) ? 2 : (W <= 3 ? 4 : 6);
};

// Home slot from the low 32 hash bits by multiplicative range reduction (any
// table size below 2^32); the fingerprint comes from the high 32 bits.
__device__ __forceinline__ uint64_t slot_home(uint64_t h, uint64_t slots)
{
    return ((h & 0xFFFFFFFFull) * slots) >> 32;
}

__device__ __forceinline__ uint64_t slot_next(uint64_t pos, uint64_t slots)
{
    return pos + 1 == slots ? 0 : pos + 1;
}

template <int W>
__device__ __forceinline__ uint32_t fingerprint(uint64_t h)
{
    uint32_t f = (uint32_t)(h >> 32);
    return f == 0xFFFFFFFFu ? 0xFFFFFFFEu : f;
}

// 16-byte compare-and-swap (PTX atom.cas.b128, sm_90 and later) of an aligned
// pair of words; returns the previous contents in old_lo, old_hi.
__device__ __forceinline__ void cas128(uint64_t* p, uint64_t cmp_lo, uint64_t cmp_hi, uint64_t new_lo,
                                       uint64_t new_hi, uint64_t& old_lo, uint64_t& old_hi)
{
    asm volatile(
        "{\n\t"
        ".reg .b128 d, b, c;\n\t"
        "mov.b128 b, {%2, %3};\n\t"
        "mov.b128 c, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], b, c;\n\t"
        "mov.b128 {%0, %1}, d;\n\t"
        "}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(p)
        : "memory");
}

// A slot's tag and key words, read with independent 16-byte loads (a slot of
// kWords 64-bit words is 16-byte aligned), so that a probe is one round trip.
template <int W>
struct SlotVal {
    uint64_t w[Slot<W>::kWords];
};

// RO: the table does not change while the kernel runs (the read-only path
// may then keep a probed line in L1 for the next slot of the probe).
template <int W, bool RO>
__device__ __forceinline__ SlotVal<W> read_slot(const uint64_t* __restrict__ sl)
{
    SlotVal<W> v;
#pragma unroll
    for (int i = 0; i < Slot<W>::kWords / 2; ++i) {
        const ulonglong2* a = reinterpret_cast<const ulonglong2*>(sl) + i;
        const ulonglong2 p = RO ? __ldg(a) : __ldcg(a);
        v.w[2 * i] = p.x;
        v.w[2 * i + 1] = p.y;
    }
    return v;
}

template <int W>
__device__ __forceinline__ bool slot_has_key(const SlotVal<W>& v, const Key<W>& key)
{
    bool eq = true;
#pragma unroll
    for (int i = 0; i < W; ++i) eq &= (v.w[1 + i] == key.w[i]);
    return eq;
}

// Read-only lookup in a table whose entries are final (every slot holds a
// row's tag and key): row of key or -1.
template <int W>
__device__ __forceinline__ int64_t table_lookup(const uint64_t* __restrict__ table, uint64_t slots,
                                                const Key<W>& key)
{
    uint64_t h = key_hash<W>(key);
    uint64_t fp = fingerprint<W>(h);
    uint64_t pos = slot_home(h, slots);
    for (uint32_t probe = 0; probe < kMaxProbe; ++probe) {
        const SlotVal<W> v = read_slot<W, true>(table + pos * Slot<W>::kWords);
        if (v.w[0] == kEmpty) return -1;
        if ((v.w[0] >> 32) == fp && slot_has_key<W>(v, key)) return (int64_t)(uint32_t)v.w[0];
        pos = slot_next(pos, slots);
    }
    return -1;
}

// Insert a unique row key (no duplicates possible): claim the first empty slot.
template <int W>
__device__ __forceinline__ bool table_insert_unique(uint64_t* table, uint64_t slots, const Key<W>& key,
                                                    uint32_t row)
{
    uint64_t h = key_hash<W>(key);
    uint64_t tag = ((uint64_t)fingerprint<W>(h) << 32) | row;
    uint64_t pos = slot_home(h, slots);
    for (uint32_t probe = 0; probe < kMaxProbe; ++probe) {
        uint64_t* sl = table + pos * Slot<W>::kWords;
        if (__ldcg(sl) == kEmpty) {
            unsigned long long old = atomicCAS((unsigned long long*)sl, kEmpty, tag);
            if (old == kEmpty) {
#pragma unroll
                for (int i = 0; i < W; ++i) sl[1 + i] = key.w[i];
                return true;
            }
        }
        pos = slot_next(pos, slots);
    }
    return false;
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; *total gets the sum.
template <int BLOCK>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    __shared__ uint32_t ws[BLOCK / 32];
    __shared__ uint32_t tot;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = lane < BLOCK / 32 ? ws[lane] : 0u;
        uint32_t xi = warp_incl_scan(x);
        if (lane < BLOCK / 32) ws[lane] = xi - x;
        if (lane == 31) tot = xi;
    }
    __syncthreads();
    uint32_t r = ws[warp] + inc - v;
    *total = tot;
    __syncthreads();
    return r;
}

// Deterministic block sum of several doubles (fixed shuffle tree + fixed warp order).
template <int BLOCK, int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* out /* smem or global, K values */)
{
    __shared__ double red[BLOCK / 32][K];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < BLOCK / 32; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// |v| 2^(32 - L) as an FP32 number, from the upper 32 bits of the FP64 v (20
// bits of significand, truncated: relative error below 2^-20), with integer
// operations only, so that magnitude tests cost the FP64 pipe nothing.
// Results below 2^-126 give 0 or a subnormal; results at or above 2^128
// saturate near 2^128.
__device__ __forceinline__ float mag_scaled_f32(double v, int L)
{
    int h = __double2hiint(v) & 0x7FFFFFFF;
    int e = (h >> 20) - (1023 - 127 - 32) - L;
    e = min(max(e, 0), 254);
    return __int_as_float((e << 23) | ((h & 0xFFFFF) << 3));
}

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;   // 20 s

}  // namespace paces
