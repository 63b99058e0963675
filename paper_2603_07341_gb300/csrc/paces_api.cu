// paces_api.cu -- host runtime behind include/paces.h: model tables, key layout,
// device memory through the caller's allocator, the step driver (stage kernels
// enqueued back to back on one stream, device-side error word checked once per
// chunk of steps), automatic capacity growth, and the export calls.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "paces.h"
#include "runtime.h"

using namespace paces;

namespace {

constexpr int kChunk = 8;                 // steps enqueued between error checks
constexpr uint32_t kMinRows = 1u << 10;
constexpr uint32_t kDefaultRows = 1u << 16;
constexpr uint64_t kMaxRowsHard = (1ull << 30) - 1;   // table slots (2 cap + 1) stay below 2^31

struct Stage {
    enum { Trunc = 0, Expand = 1, Csr = 2, Taylor = 3, Obs = 4, Other = 5 };
};

uint64_t next_pow2(uint64_t v)
{
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

UDiv make_udiv(uint64_t d)
{
    UDiv u;
    u.d = d;
    int l = 0;
    while (l < 64 && (((unsigned __int128)1) << l) < d) ++l;          // l = ceil(log2 d)
    unsigned __int128 two64 = ((unsigned __int128)1) << 64;
    unsigned __int128 twol = ((unsigned __int128)1) << l;
    u.m = (uint64_t)((two64 * (twol - d)) / d + 1);
    u.sh1 = l < 1 ? (uint32_t)l : 1u;
    u.sh2 = l > 1 ? (uint32_t)(l - 1) : 0u;
    return u;
}

struct DevAlloc {
    void* p;
    size_t bytes;
};

}  // namespace

struct paces_handle {
    paces_params prm;
    std::vector<double> eps, omega, g, Jx;
    std::vector<int32_t> cap;
    paces_layout lay;
    DevModel* hmodel = nullptr;   // host copy
    int W = 1, D = 4, P = 4, N = 1, lpr = 1, R = 1;
    int table_pct = 50;                    // largest hash-table load, percent
    paces_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t st = nullptr;
    int device = 0, sms = 1;
    std::string err;

    Bufs b{};
    std::vector<DevAlloc> row_allocs;      // freed on growth
    std::vector<DevAlloc> fixed_allocs;    // model, counters, obs, psi0
    Counters* hctr = nullptr;              // pinned host mirror
    uint32_t cap_rows = 0;

    int gen = 0;
    bool fresh = false, has_state = false, csr_valid = false;
    bool last_truncated = false;
    double time = 0.0;
    int64_t n_records = 0, obs_cap = 0;
    int64_t step_index = 0;
    int64_t psi0_cap = 0;

    bool use_graphs = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool gvalid[2] = {false, false};
    double g_dt = 0.0, g_th2 = -1.0;
    int64_t g_nom = 0;
    uint64_t g_seed = 0;
    int64_t graph_launches[PACES_NUM_STAGES + 1] = {0};

    // recording for the reverse pass: a checkpoint of the state every
    // rec_every steps, plus dt and theta^2 of every recorded step
    struct Ckpt {
        int64_t step;             // recorded step that starts from this state
        uint32_t q;
        bool fresh;
        double time;
        DevAlloc mem;             // keys | meta | amplitudes
    };
    int rec_every = 0;
    bool rec_valid = false;
    int64_t rec_steps = 0, rec_base = 0;   // rec_base: record written by recorded step 0
    std::vector<double> rec_dt, rec_th2;
    std::vector<int64_t> rec_nom;            // top-q_nom truncation (0: threshold)
    std::vector<uint64_t> rec_seed;
    std::vector<Ckpt> ckpts;

    bool profiling = false;
    double stage_ms[PACES_NUM_STAGES] = {0};
    double stage_bytes[PACES_NUM_STAGES] = {0};
    int64_t stage_launch[PACES_NUM_STAGES + 1] = {0};
    std::vector<cudaEvent_t> evpool;
};

namespace {

paces_status fail(paces_t h, paces_status s, const std::string& msg)
{
    if (h) h->err = msg;
    return s;
}

paces_status cuda_fail(paces_t h, cudaError_t e, const char* where)
{
    return fail(h, PACES_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(h, call)                                                  \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);           \
    } while (0)

void* dev_alloc(paces_t h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->st);
    } else if (cudaMallocAsync(&p, bytes, h->st) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(paces_t h, DevAlloc a)
{
    if (!a.p) return;
    if (h->has_alloc) h->alloc.free(h->alloc.ctx, a.p, a.bytes, (void*)h->st);
    else cudaFreeAsync(a.p, h->st);
}

template <typename T>
T* alloc_track(paces_t h, std::vector<DevAlloc>& v, size_t count)
{
    size_t bytes = ((sizeof(T) * count) + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void* p = dev_alloc(h, bytes);
    if (p) v.push_back({p, bytes});
    return (T*)p;
}

// ---------------------------------------------------------------- model tables
double hop_pattern(const paces_params& p, const std::vector<double>& Jx, int a, int b)
{
    int N = p.n_sites;
    if (a == b) return 0.0;
    if (p.lattice_kind == PACES_EXPLICIT) return Jx[(size_t)a * N + b];
    if (p.lattice_kind == PACES_RING) {
        if (N < 2) return 0.0;
        return ((a + 1) % N == b || (b + 1) % N == a) ? 1.0 : 0.0;
    }
    int d0 = N, d1 = 1;
    if (p.lattice_kind == PACES_OPEN2D || p.lattice_kind == PACES_OPEN3D) {
        d0 = p.dims[0];
        d1 = p.dims[1];
    }
    int ax = a % d0, ay = (a / d0) % d1, az = a / (d0 * d1);
    int bx = b % d0, by = (b / d0) % d1, bz = b / (d0 * d1);
    double dx = ax - bx, dy = ay - by, dz = az - bz;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (p.coupling_kind == PACES_NEAREST) return r2 == 1.0 ? 1.0 : 0.0;
    return 1.0 / (r2 * std::sqrt(r2));
}

paces_status check_params(const paces_params* p, std::string& why)
{
    if (!p) { why = "params is NULL"; return PACES_ERR_INVALID; }
    int N = p->n_sites;
    if (N < 1 || N > PACES_MAX_SITES) { why = "n_sites out of range"; return PACES_ERR_INVALID; }
    if (p->lattice_kind < 0 || p->lattice_kind > 4) { why = "lattice_kind"; return PACES_ERR_INVALID; }
    if (p->coupling_kind < 0 || p->coupling_kind > 1) { why = "coupling_kind"; return PACES_ERR_INVALID; }
    if (p->lattice_kind == PACES_RING && p->coupling_kind != PACES_NEAREST) {
        why = "a ring has nearest-neighbour coupling only";
        return PACES_ERR_INVALID;
    }
    if (p->lattice_kind == PACES_OPEN2D && (p->dims[0] < 1 || p->dims[1] < 1 || p->dims[0] * p->dims[1] != N)) {
        why = "dims[0]*dims[1] must equal n_sites";
        return PACES_ERR_INVALID;
    }
    if (p->lattice_kind == PACES_OPEN3D &&
        (p->dims[0] < 1 || p->dims[1] < 1 || p->dims[2] < 1 || p->dims[0] * p->dims[1] * p->dims[2] != N)) {
        why = "dims[0]*dims[1]*dims[2] must equal n_sites";
        return PACES_ERR_INVALID;
    }
    if (p->lattice_kind == PACES_EXPLICIT && !p->J_explicit) { why = "J_explicit is NULL"; return PACES_ERR_INVALID; }
    if (!p->phonon_cap) { why = "phonon_cap is NULL"; return PACES_ERR_INVALID; }
    for (int j = 0; j < N; ++j)
        if (p->phonon_cap[j] < 0 || p->phonon_cap[j] > kMaxCap) { why = "phonon_cap out of range"; return PACES_ERR_INVALID; }
    if (p->m < 0) { why = "m < 0"; return PACES_ERR_INVALID; }
    if (p->precision != PACES_DW && p->precision != PACES_C128 && p->precision != PACES_C64_SPMV) {
        why = "precision";
        return PACES_ERR_INVALID;
    }
    if (p->taylor_tol < 0 || p->taylor_nmax < 0 || p->fixed_terms < 0) { why = "series limits"; return PACES_ERR_INVALID; }
    if (p->batch < 0 || p->batch > PACES_MAX_BATCH) { why = "batch out of range"; return PACES_ERR_INVALID; }
    if (!std::isfinite(p->taylor_xmax)) { why = "taylor_xmax"; return PACES_ERR_INVALID; }
    if (p->propagator != PACES_TAYLOR && p->propagator != PACES_LANCZOS) { why = "propagator"; return PACES_ERR_INVALID; }
    if (p->krylov_max < 0 || p->krylov_max > PACES_MAX_KRYLOV) { why = "krylov_max"; return PACES_ERR_INVALID; }
    if (p->propagator == PACES_LANCZOS && (p->precision != PACES_C128 || p->batch > 1)) {
        why = "the Lanczos propagator needs PACES_C128 and batch <= 1";
        return PACES_ERR_INVALID;
    }
    return PACES_OK;
}

paces_status plan(const paces_params* p, paces_layout* L, std::string& why)
{
    paces_status s = check_params(p, why);
    if (s) return s;
    int N = p->n_sites;
    const unsigned __int128 lim = (((unsigned __int128)1) << 64) - 1;   // keep the all-ones key invalid
    paces_layout cand[2];
    for (int mode = 0; mode < 2; ++mode) {       // 0: power-of-two radices, 1: dense
        paces_layout& l = cand[mode];
        std::memset(&l, 0, sizeof(l));
        l.n_sites = N;
        l.pow2 = mode == 0;
        l.exciton_radix = mode == 0 ? next_pow2((uint64_t)N) : (uint64_t)N;
        int w = 0;
        unsigned __int128 prod = l.exciton_radix;
        for (int j = 0; j < N; ++j) {
            uint64_t r = (uint64_t)p->phonon_cap[j] + 1;
            if (mode == 0) r = next_pow2(r);
            if (prod * r > lim) {
                ++w;
                prod = 1;
            }
            l.site_word[j] = w;
            l.site_stride[j] = (uint64_t)prod;
            l.site_radix[j] = r;
            prod *= r;
        }
        uint64_t rb = (uint64_t)(p->batch > 1 ? p->batch : 1);
        if (mode == 0) rb = next_pow2(rb);
        if (prod * rb > lim) {
            ++w;
            prod = 1;
        }
        l.batch_word = w;
        l.batch_stride = (uint64_t)prod;
        l.batch_radix = rb;
        l.words = w + 1;
    }
    *L = cand[0].words <= cand[1].words ? cand[0] : cand[1];
    if (L->words > PACES_MAX_WORDS) {
        why = "the basis needs " + std::to_string(L->words) + " 64-bit words";
        return PACES_ERR_KEY_WIDTH;
    }
    return PACES_OK;
}

paces_status encode(const paces_layout* L, int64_t n, const int32_t* site, const int32_t* occ, uint64_t* keys,
                    std::string& why)
{
    int N = L->n_sites, W = L->words;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t* k = keys + i * W;
        for (int w = 0; w < W; ++w) k[w] = 0;
        if (site[i] < 0 || site[i] >= N) { why = "site out of range"; return PACES_ERR_INVALID; }
        k[0] = (uint64_t)site[i];
        for (int j = 0; j < N; ++j) {
            int32_t v = occ[i * N + j];
            uint64_t cap = L->site_radix[j];
            if (v < 0 || (uint64_t)v >= cap) { why = "occupation out of range"; return PACES_ERR_INVALID; }
            k[L->site_word[j]] += (uint64_t)v * L->site_stride[j];
        }
    }
    return PACES_OK;
}

// ---------------------------------------------------------------- buffers
size_t slot_words(int W) { return W == 1 ? 2 : (W <= 3 ? 4 : 6); }

void free_rows(paces_t h)
{
    for (auto& a : h->row_allocs) dev_free(h, a);
    h->row_allocs.clear();
}

// Krylov vectors the Lanczos propagator may hold per series.
int krylov_dim(paces_t h) { return h->prm.krylov_max > 0 ? h->prm.krylov_max : 30; }

// Key of the propagator kernel for occupancy queries.
int prop_key(paces_t h) { return h->prm.propagator == PACES_LANCZOS ? kPrecLanczos : h->prm.precision; }

// Allocate every row-sized buffer for cap rows; on failure frees what it got.

paces_status alloc_rows(paces_t h, uint32_t cap, std::vector<DevAlloc>& out, Bufs& b)
{
    std::vector<DevAlloc> saved;
    saved.swap(h->row_allocs);
    // load factor <= table_pct / 100; slot indices must stay below 2^31 (a
    // candidate slot shares its 32-bit word with the kCand flag)
    uint64_t slots = (uint64_t)cap * 100 / (uint64_t)h->table_pct + 1;
    if (slots >= (1ull << 31)) return PACES_ERR_CAPACITY;
    size_t sw = slot_words(h->W);
    bool ok = true;
    auto chk = [&](void* p) { ok = ok && p; };
    for (int g = 0; g < 2; ++g) {
        chk(b.keys[g] = alloc_track<uint64_t>(h, h->row_allocs, (size_t)cap * h->W));
        chk(b.meta[g] = alloc_track<uint32_t>(h, h->row_allocs, cap));
        chk(b.table[g] = alloc_track<uint64_t>(h, h->row_allocs, slots * sw));
    }
    for (int v = 0; v < 4; ++v) chk(b.V[v] = alloc_track<double2>(h, h->row_allocs, cap));
    if (h->prm.precision == PACES_C64_SPMV) {
        for (int v = 0; v < 2; ++v) chk(b.F[v] = alloc_track<float2>(h, h->row_allocs, cap));
    } else {
        b.F[0] = b.F[1] = nullptr;
    }
    chk(b.col = alloc_track<uint32_t>(h, h->row_allocs, (size_t)cap * h->P));
    chk(b.cid = alloc_track<uint8_t>(h, h->row_allocs, (size_t)cap * h->P));
    chk(b.cnt = alloc_track<uint8_t>(h, h->row_allocs, cap));
    chk(b.diag = alloc_track<double>(h, h->row_allocs, cap));
    if (h->prm.precision == PACES_C128) {
        chk(b.diag_h = alloc_track<double>(h, h->row_allocs, cap));
        chk(b.rperm = alloc_track<uint8_t>(h, h->row_allocs, (size_t)cap + kBlock));
    } else {
        b.diag_h = nullptr;
        b.rperm = nullptr;
    }
    chk(b.cand_slot = alloc_track<uint32_t>(h, h->row_allocs, (size_t)cap * h->D));
    if (h->prm.propagator == PACES_LANCZOS)
        chk(b.kry = alloc_track<double2>(h, h->row_allocs, (size_t)cap * krylov_dim(h)));
    else
        b.kry = nullptr;
    // sort of the kept set: indices in the winner-mask buffer (free during
    // truncation); keys in the two term buffers when a key fits in 16 bytes
    if (h->W <= 2) {
        b.sortk[0] = reinterpret_cast<uint64_t*>(b.V[2]);
        b.sortk[1] = reinterpret_cast<uint64_t*>(b.V[3]);
    } else {
        for (int s = 0; s < 2; ++s) chk(b.sortk[s] = alloc_track<uint64_t>(h, h->row_allocs, (size_t)cap * h->W));
    }
    chk(b.masks = alloc_track<uint64_t>(h, h->row_allocs, cap));
    b.sorti[0] = reinterpret_cast<uint32_t*>(b.masks);
    b.sorti[1] = reinterpret_cast<uint32_t*>(b.masks) + cap;
    chk(b.keepw = alloc_track<uint32_t>(h, h->row_allocs, cap / 32 + 64));
    out.swap(h->row_allocs);
    h->row_allocs.swap(saved);
    if (!ok) {
        for (auto& a : out) dev_free(h, a);
        out.clear();
        return PACES_ERR_CAPACITY;
    }
    b.table_slots = slots;
    b.cap_rows = cap;
    b.cand_cap = (uint64_t)cap * h->D;
    return PACES_OK;
}

paces_status set_counters(paces_t h)
{
    CUDA_TRY(h, cudaMemcpyAsync(h->b.ctr, h->hctr, sizeof(Counters), cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    return PACES_OK;
}

paces_status read_counters(paces_t h)
{
    CUDA_TRY(h, cudaMemcpyAsync(h->hctr, h->b.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    return PACES_OK;
}

void count(paces_t h, int stage, int n)
{
    if (n > 0) h->stage_launch[stage] += n;
}

paces_status clear_table(paces_t h, int gen)
{
    CUDA_TRY(h, cudaMemsetAsync(h->b.table[gen], 0xFF, h->b.table_slots * slot_words(h->W) * 8, h->st));
    return PACES_OK;
}

void invalidate_graphs(paces_t h)
{
    for (int g = 0; g < 2; ++g) {
        if (h->gexec[g]) cudaGraphExecDestroy(h->gexec[g]);
        h->gexec[g] = nullptr;
        h->gvalid[g] = false;
    }
}

// Grow the row capacity to at least `want`, keeping the current state (rows
// [0, q) of generation gen in keys and in vector V[vec]) and rebuilding its
// table.  Only the live state is stashed while the old buffers are released,
// so the new capacity may use nearly all of the device memory.  Growth tries
// 2x, then 1.5x, then 1.25x, then exactly `want`.
paces_status grow(paces_t h, uint64_t want, uint32_t q, int vec)
{
    uint64_t cur = h->cap_rows, base = std::max<uint64_t>(cur, kMinRows);
    if (want > kMaxRowsHard) return fail(h, PACES_ERR_CAPACITY, "more than 2^30 - 1 rows (table slot indices use 31 bits)");
    uint64_t* sk = nullptr;
    double2* sv = nullptr;
    uint32_t* sm = nullptr;
    size_t kb = (size_t)q * h->W * 8, vb = (size_t)q * sizeof(double2), mb = (size_t)q * 4;
    if (q > 0 && cur > 0) {
        sk = (uint64_t*)dev_alloc(h, kb);
        sv = (double2*)dev_alloc(h, vb);
        sm = (uint32_t*)dev_alloc(h, mb);
        if (!sk || !sv || !sm) {
            if (sk) dev_free(h, {sk, kb});
            if (sv) dev_free(h, {sv, vb});
            if (sm) dev_free(h, {sm, mb});
            return fail(h, PACES_ERR_CAPACITY, "no room to stash the state while growing");
        }
        CUDA_TRY(h, cudaMemcpyAsync(sk, h->b.keys[h->gen], kb, cudaMemcpyDeviceToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync(sv, h->b.V[vec], vb, cudaMemcpyDeviceToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync(sm, h->b.meta[h->gen], mb, cudaMemcpyDeviceToDevice, h->st));
    }
    free_rows(h);
    Bufs nb = h->b;
    std::vector<DevAlloc> na;
    uint64_t tries[5] = {base * 2, base + base / 2, base + base / 4, want, cur};
    uint64_t got = 0;
    for (int t = 0; t < 5 && !got; ++t) {
        uint64_t cap = std::min<uint64_t>(std::max<uint64_t>(tries[t], t < 4 ? want : 0), kMaxRowsHard);
        if (cap == 0 || (t == 4 && cap < q)) continue;
        if (alloc_rows(h, (uint32_t)cap, na, nb) == PACES_OK) got = cap;
    }
    if (!got) {
        if (sk) dev_free(h, {sk, kb});
        if (sv) dev_free(h, {sv, vb});
        if (sm) dev_free(h, {sm, mb});
        h->has_state = false;
        return fail(h, PACES_ERR_CAPACITY, "device allocation failed; the state was lost");
    }
    h->row_allocs.swap(na);
    h->b = nb;
    h->cap_rows = (uint32_t)got;
    invalidate_graphs(h);
    if (sk) {
        CUDA_TRY(h, cudaMemcpyAsync(h->b.keys[h->gen], sk, kb, cudaMemcpyDeviceToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync(h->b.V[vec], sv, vb, cudaMemcpyDeviceToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync(h->b.meta[h->gen], sm, mb, cudaMemcpyDeviceToDevice, h->st));
        dev_free(h, {sk, kb});
        dev_free(h, {sv, vb});
        dev_free(h, {sm, mb});
    }
    paces_status s = clear_table(h, h->gen);
    if (s) return s;
    if (q > 0) count(h, Stage::Other, launch_insert_rows(h->b, h->gen, q, h->st));
    CUDA_TRY(h, cudaGetLastError());
    if (got < want) return fail(h, PACES_ERR_CAPACITY, "device memory exhausted at " + std::to_string(got) + " rows");
    return PACES_OK;
}

paces_status ensure_obs(paces_t h, int64_t need)
{
    if (need <= h->obs_cap) return PACES_OK;
    int64_t ncap = std::max<int64_t>(need, std::max<int64_t>(64, 2 * h->obs_cap));
    size_t rl = (size_t)h->b.rec_len;
    double* nb = (double*)dev_alloc(h, sizeof(double) * rl * ncap);
    if (!nb) return fail(h, PACES_ERR_CAPACITY, "observables buffer");
    CUDA_TRY(h, cudaMemsetAsync(nb, 0, sizeof(double) * rl * ncap, h->st));
    if (h->b.obs) {
        if (h->n_records > 0)
            CUDA_TRY(h, cudaMemcpyAsync(nb, h->b.obs, sizeof(double) * rl * h->n_records, cudaMemcpyDeviceToDevice,
                                        h->st));
        for (auto it = h->fixed_allocs.begin(); it != h->fixed_allocs.end(); ++it)
            if (it->p == h->b.obs) {
                dev_free(h, *it);
                h->fixed_allocs.erase(it);
                break;
            }
    }
    h->fixed_allocs.push_back({nb, sizeof(double) * rl * ncap});
    h->b.obs = nb;
    h->obs_cap = ncap;
    invalidate_graphs(h);
    return PACES_OK;
}

TaylorParams taylor_params(paces_t h, double dt, int step)
{
    TaylorParams p;
    p.dt = dt;
    double tol = h->prm.taylor_tol > 0 ? h->prm.taylor_tol : 1e-15;
    p.tol2 = tol * tol;
    p.nmax = h->prm.taylor_nmax > 0 ? h->prm.taylor_nmax : 200;
    p.fixed_terms = h->prm.fixed_terms;
    p.xmax = h->prm.taylor_xmax == 0.0 ? 8.0 : (h->prm.taylor_xmax < 0.0 ? 0.0 : h->prm.taylor_xmax);
    p.step = step;
    p.lpr = h->lpr;
    p.c64 = h->prm.precision == PACES_C64_SPMV;
    p.fmt = h->b.fmt;
    p.lanczos = h->prm.propagator == PACES_LANCZOS;
    p.kmax = krylov_dim(h);
    return p;
}

cudaEvent_t ev(paces_t h, size_t i)
{
    while (h->evpool.size() <= i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->evpool.push_back(e);
    }
    return h->evpool[i];
}

// Enqueue the kernels of one time step on stream st, reading generation gin
// (fresh: the state set by set_state, no truncation).  Touches no host state
// except launch counts, so it can be captured into a CUDA graph.  Returns the
// output generation.  ev_base: first of 6 events (profiling only).
int enqueue_kernels(paces_t h, cudaStream_t st, int gin, bool fresh, double dt, double th2, int64_t q_nom,
                    uint64_t seed, int step,
                    bool prof, size_t ev_base)
{
    const Bufs& b = h->b;
    auto mark = [&](int k) {
        if (prof) cudaEventRecord(ev(h, ev_base + k), st);
    };
    mark(0);
    int gen = gin;
    if (!fresh) {
        int gout = 1 - gin;
        cudaMemsetAsync(b.table[gout], 0xFF, b.table_slots * slot_words(h->W) * 8, st);
        if (q_nom > 0) count(h, Stage::Trunc, launch_truncate_nom(b, gin, gout, (uint64_t)q_nom, seed, step, st));
        else count(h, Stage::Trunc, launch_truncate(b, gin, gout, th2, step, st));
        mark(1);
        for (int f = 0; f < h->prm.m; ++f) count(h, Stage::Expand, launch_level(b, gout, f, gin, step, st));
        gen = gout;
    } else {
        mark(1);
    }
    mark(2);
    count(h, Stage::Csr, launch_csr(b, gen, st));
    mark(3);
    count(h, Stage::Taylor, launch_taylor(b, taylor_params(h, dt, step), st));
    mark(4);
    count(h, Stage::Obs, launch_observe(b, gen, b.V[0], dt, fresh ? 2 : 0, st));
    mark(5);
    return gen;
}

void enqueue_step(paces_t h, double dt, double th2, int64_t q_nom, uint64_t seed, size_t ev_base)
{
    int step = (int)(h->step_index & 0x7fffffff);
    bool fresh = h->fresh;
    int gen = -1;
    if (!fresh && h->use_graphs && !h->profiling) {
        int gin = h->gen;
        if (!h->gvalid[gin] || h->g_dt != dt || h->g_th2 != th2 || h->g_nom != q_nom || h->g_seed != seed) {
            if (h->gexec[gin]) cudaGraphExecDestroy(h->gexec[gin]);
            h->gexec[gin] = nullptr;
            h->gvalid[gin] = false;
            if (!h->cap_stream) cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
            cudaGraph_t g = nullptr;
            int64_t saved[PACES_NUM_STAGES + 1];
            std::memcpy(saved, h->stage_launch, sizeof(saved));
            bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) enqueue_kernels(h, h->cap_stream, gin, false, dt, th2, q_nom, seed, step, false, 0);
            ok = cudaStreamEndCapture(h->cap_stream, &g) == cudaSuccess && ok;
            std::memcpy(h->graph_launches, h->stage_launch, sizeof(saved));
            for (int i = 0; i <= PACES_NUM_STAGES; ++i) h->graph_launches[i] -= saved[i];
            std::memcpy(h->stage_launch, saved, sizeof(saved));
            if (ok) ok = cudaGraphInstantiate(&h->gexec[gin], g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (!ok) {                    // capture unavailable: launch directly from now on
                h->use_graphs = false;
                h->gexec[gin] = nullptr;
            } else {
                h->gvalid[gin] = true;
                h->g_dt = dt;
                h->g_th2 = th2;
                h->g_nom = q_nom;
                h->g_seed = seed;
            }
        }
        if (h->gvalid[gin]) {
            cudaGraphLaunch(h->gexec[gin], h->st);
            for (int i = 0; i <= PACES_NUM_STAGES; ++i) h->stage_launch[i] += h->graph_launches[i];
            gen = 1 - gin;
        }
    }
    if (gen < 0) gen = enqueue_kernels(h, h->st, h->gen, fresh, dt, th2, q_nom, seed, step, h->profiling, ev_base);
    h->last_truncated = !fresh;
    h->gen = gen;
    h->fresh = false;
    h->csr_valid = true;
    h->step_index += 1;
}


// ---------------------------------------------------------------- recording
void drop_recording(paces_t h)
{
    for (auto& c : h->ckpts) dev_free(h, c.mem);
    h->ckpts.clear();
    h->rec_dt.clear();
    h->rec_th2.clear();
    h->rec_nom.clear();
    h->rec_seed.clear();
    h->rec_steps = 0;
    h->rec_valid = h->rec_every > 0;
    h->rec_base = h->n_records;
}

size_t state_bytes(paces_t h, uint32_t q, size_t* off_meta, size_t* off_vec)
{
    size_t kb = ((size_t)q * h->W * 8 + 255) & ~(size_t)255;
    size_t mb = ((size_t)q * 4 + 255) & ~(size_t)255;
    *off_meta = kb;
    *off_vec = kb + mb;
    return kb + mb + (size_t)q * 16 + 256;
}

// Copy rows [0, q) of generation gen (keys, meta, amplitudes of V[vec]) to dst.
paces_status copy_state_out(paces_t h, int gen, int vec, uint32_t q, char* dst)
{
    size_t om, ov;
    state_bytes(h, q, &om, &ov);
    if (q == 0) return PACES_OK;
    CUDA_TRY(h, cudaMemcpyAsync(dst, h->b.keys[gen], (size_t)q * h->W * 8, cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(dst + om, h->b.meta[gen], (size_t)q * 4, cudaMemcpyDeviceToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(dst + ov, h->b.V[vec], (size_t)q * 16, cudaMemcpyDeviceToDevice, h->st));
    return PACES_OK;
}

// Make a copied state the live one (generation 0; V1 when fresh, else V0),
// with its table rebuilt and one BFS level, so that a P H P build uses table
// lookups for every row.
paces_status restore_state(paces_t h, const char* src, uint32_t q, bool fresh, double time, int64_t rec_index,
                           const Counters* base = nullptr)
{
    size_t om, ov;
    state_bytes(h, q, &om, &ov);
    int vec = fresh ? 1 : 0;
    h->gen = 0;
    paces_status s = clear_table(h, 0);
    if (s) return s;
    if (q > 0) {
        CUDA_TRY(h, cudaMemcpyAsync(h->b.keys[0], src, (size_t)q * h->W * 8, cudaMemcpyDeviceToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync(h->b.meta[0], src + om, (size_t)q * 4, cudaMemcpyDeviceToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync(h->b.V[vec], src + ov, (size_t)q * 16, cudaMemcpyDeviceToDevice, h->st));
        count(h, Stage::Other, launch_insert_rows(h->b, 0, q, h->st));
    }
    if (base) *h->hctr = *base;
    else std::memset(h->hctr, 0, sizeof(Counters));
    h->hctr->q = q;
    h->hctr->q_in = q;
    h->hctr->kept = q;
    h->hctr->level_off[0] = 0;
    h->hctr->level_off[1] = q;
    h->hctr->nlevels = 1;
    h->hctr->time = time;
    h->hctr->rec_index = (uint32_t)rec_index;
    h->hctr->err = 0;
    s = set_counters(h);
    if (s) return s;
    h->fresh = fresh;
    return PACES_OK;
}

// Checkpoint the live state before recorded step h->rec_steps.
paces_status save_checkpoint(paces_t h)
{
    if (!h->ckpts.empty() && h->ckpts.back().step == h->rec_steps) return PACES_OK;
    uint32_t q = h->hctr->q;
    size_t om, ov, bytes = state_bytes(h, q, &om, &ov);
    void* p = dev_alloc(h, bytes);
    if (!p) return fail(h, PACES_ERR_CAPACITY, "checkpoint buffer");
    bytes = (bytes + 255) & ~(size_t)255;
    paces_handle::Ckpt c{h->rec_steps, q, h->fresh, h->hctr->time, {p, bytes}};
    paces_status s = copy_state_out(h, h->gen, h->fresh ? 1 : 0, q, (char*)p);
    if (s) {
        dev_free(h, c.mem);
        return s;
    }
    h->ckpts.push_back(c);
    return PACES_OK;
}


// Algorithmic bytes of one step from its record (the per-unit figures stated
// at paces_stage_stats); fills bytes[5].
void step_bytes(paces_t h, const double* r, double q_in, bool truncated, double* bytes)
{
    double W8 = 8.0 * h->W, q = r[PACES_OBS_ROWS], kept = r[PACES_OBS_KEPT];
    double nnz_off = r[PACES_OBS_NNZ] - q, terms = r[PACES_OBS_TERMS];
    double slot = 8.0 * slot_words(h->W);
    if (truncated) {
        bytes[0] += q_in * (16.0 + 0.25) + kept * (2.0 * (W8 + 16.0) + slot);
        // every row is a frontier row once: key read twice, D candidate slots
        // written and read, its winner mask written and read; each new row: key,
        // table slot, one rescue probe sector, c'
        double newrows = q - kept;
        bytes[1] += q * (2.0 * W8 + 8.0 * h->D + 16.0) + newrows * (W8 + slot + 32.0 + 16.0);
    }
    bytes[2] += q * (W8 + 9.0) + nnz_off * 5.0 + q * h->D * 32.0;
    if (h->prm.propagator == PACES_LANCZOS) {
        // per Krylov vector: pass A 1 + 8 + 16 (s_j) + 16 (t) per row and 5 per
        // entry, pass B 3 x 16 read + 16 written; per series the combination
        // reads its n vectors and writes r
        double nsub = r[PACES_OBS_SUBSTEPS];
        bytes[3] += terms * (q * 105.0 + nnz_off * 5.0) + q * 16.0 * (terms + nsub);
    } else if (terms >= 1) {
        bytes[3] += q * 57.0 + nnz_off * 5.0 + (terms - 1) * (q * 73.0 + nnz_off * 5.0);
    }
    bytes[4] += q * (W8 + 16.0);
}

}  // namespace

// Device-side description of a model (bond lists in canonical move order,
// coefficient table, key-layout divisors), built on the host from params.
paces_status paces::fill_model(const paces_params* params, const paces_layout& L, DevModel* M)
{
    const int N = params->n_sites;
    std::vector<double> Jx;
    if (params->lattice_kind == PACES_EXPLICIT) Jx.assign(params->J_explicit, params->J_explicit + (size_t)N * N);
    auto at = [](const double* v, int j) { return v ? v[j] : 0.0; };
    std::memset(M, 0, sizeof(DevModel));
    M->N = N;
    M->W = L.words;
    M->pow2 = L.pow2;
    M->div_exc = make_udiv(L.exciton_radix);
    int w = 0;
    M->word_first[0] = 0;
    for (int j = 0; j < N; ++j) {
        while (L.site_word[j] > w) M->word_first[++w] = j;
        M->site_word[j] = L.site_word[j];
        M->stride[j] = L.site_stride[j];
        M->div_stride[j] = make_udiv(L.site_stride[j]);
        M->div_radix[j] = make_udiv(L.site_radix[j]);
        M->cap[j] = params->phonon_cap[j];
        M->gnz[j] = at(params->g, j) != 0.0;
        M->eps[j] = at(params->eps, j);
        M->omega[j] = at(params->omega, j);
        M->eps_dw[j] = dw_from_double(M->eps[j]);
        M->omega_dw[j] = dw_from_double(M->omega[j]);
    }
    M->uniform_omega = 1;
    for (int j = 1; j < N; ++j) M->uniform_omega &= (M->omega[j] == M->omega[0]);
    M->uniform_radix = 1;
    for (int j = 1; j < N; ++j) M->uniform_radix &= (L.site_radix[j] == L.site_radix[0]);
    M->r8_ok = 0;
    if (M->uniform_radix && L.words == 1 && N <= 16 && L.site_radix[0] >= 2) {
        const uint64_t R = L.site_radix[0];
        uint64_t r8 = 1;
        bool fits = true;
        for (int i = 0; i < 8 && fits; ++i) {
            r8 *= R;
            fits = r8 < (1ull << 32);
        }
        if (fits && r8 * (R - 1) < (1ull << 32)) {
            M->r8_ok = 1;
            M->r_magic = (uint32_t)(((1ull << 32) + R - 1) / R);
            M->div_r8 = make_udiv(r8);
        }
    }
    M->batch = params->batch > 1 ? params->batch : 1;
    M->batch_word = L.batch_word;
    M->div_batch_stride = make_udiv(L.batch_stride);
    M->div_batch_radix = make_udiv(L.batch_radix);
    M->fmt = params->precision == PACES_C128 ? 1 : 0;
    while (w < L.words) M->word_first[++w] = N;
    std::map<std::tuple<double, double, double>, int> ids;
    auto cid_of = [&](double v, double dJ, double dg) -> int {
        auto key = std::make_tuple(v, dJ, dg);
        auto it = ids.find(key);
        if (it != ids.end()) return it->second;
        int id = (int)ids.size();
        ids[key] = id;
        if (id < kMaxCoefs) {
            M->coef[id] = v;
            M->coef_dJ[id] = dJ;
            M->coef_dg[id] = dg;
        }
        return id;
    };
    int maxdeg = 0, nadj = 0, nlad = 0;
    for (int si = 0; si < N; ++si) {
        M->adj_off[si] = nadj;
        for (int t = 0; t < N; ++t) {
            double p = hop_pattern(*params, Jx, t, si);
            double v = params->J * p;
            if (t == si || v == 0.0) continue;
            if (nadj - M->adj_off[si] >= kMaxMoves - 2) return PACES_ERR_UNSUPPORTED;
            M->adj[nadj] = (uint8_t)t;
            M->adj_cid[nadj] = (uint8_t)std::min(cid_of(v, p, 0.0), 255);
            ++nadj;
        }
        maxdeg = std::max(maxdeg, nadj - M->adj_off[si]);
        M->lad_off[si] = nlad;
        for (int k = 0; k < params->phonon_cap[si]; ++k) {
            double sq = std::sqrt((double)(k + 1));
            M->lad_cid[nlad + k] = (uint8_t)std::min(cid_of(at(params->g, si) * sq, 0.0, sq), 255);
        }
        nlad += params->phonon_cap[si];
    }
    M->adj_off[N] = nadj;
    M->lad_off[N] = nlad;
    // integer row-bound tables (up20 = |x| rounded up to a multiple of 2^-20)
    auto up20 = [](double x) { return (unsigned long long)std::ceil(std::fabs(x) * 1048576.0); };
    for (int c = 0; c < (int)ids.size() && c < kMaxCoefs; ++c) M->hb_coef[c] = up20(M->coef[c]);
    for (int si = 0; si < N; ++si) {
        M->hb_eps[si] = up20(M->eps[si]);
        M->hb_omega[si] = up20(M->omega[si]);
        unsigned long long hs = 0;
        for (int e = M->adj_off[si]; e < M->adj_off[si + 1]; ++e) hs += M->hb_coef[M->adj_cid[e]];
        M->hb_hop[si] = hs;
    }
    M->nlad = nlad;
    M->ncoef = (int)ids.size();
    if (M->ncoef > kMaxCoefs) return PACES_ERR_UNSUPPORTED;
    M->D = maxdeg + 2;
    M->P = (M->D + 3) / 4 * 4;
    M->div_D = make_udiv((uint64_t)M->D);
    return PACES_OK;
}

paces_status paces::plan_layout_internal(const paces_params* params, paces_layout* out)
{
    std::string why;
    return plan(params, out, why);
}

// ======================================================================== C ABI
extern "C" {

paces_status paces_plan_layout(const paces_params* params, paces_layout* out)
{
    std::string why;
    if (!out) return PACES_ERR_INVALID;
    return plan(params, out, why);
}

paces_status paces_encode_keys(const paces_layout* layout, int64_t n, const int32_t* site, const int32_t* occ,
                               uint64_t* keys)
{
    std::string why;
    if (!layout || n < 0 || (n > 0 && (!site || !occ || !keys))) return PACES_ERR_INVALID;
    if (layout->words < 1 || layout->words > PACES_MAX_WORDS) return PACES_ERR_INVALID;
    return encode(layout, n, site, occ, keys, why);
}

paces_status paces_create(const paces_params* params, const paces_allocator* alloc, void* stream, paces_t* out)
{
    if (!out) return PACES_ERR_INVALID;
    *out = nullptr;
    std::string why;
    paces_layout L;
    paces_status s = plan(params, &L, why);
    if (s) return s;
    paces_t h = new paces_handle();
    h->prm = *params;
    int N = params->n_sites;
    h->N = N;
    h->lay = L;
    h->W = L.words;
    h->R = params->batch > 1 ? params->batch : 1;
    h->eps.assign((size_t)N * h->R, 0.0);
    h->omega.assign(N, 0.0);
    h->g.assign(N, 0.0);
    h->cap.assign(params->phonon_cap, params->phonon_cap + N);
    if (params->eps)
        for (size_t j = 0; j < h->eps.size(); ++j) h->eps[j] = params->eps[j];
    for (int j = 0; j < N; ++j) {
        if (params->omega) h->omega[j] = params->omega[j];
        if (params->g) h->g[j] = params->g[j];
    }
    if (params->lattice_kind == PACES_EXPLICIT) h->Jx.assign(params->J_explicit, params->J_explicit + (size_t)N * N);
    h->prm.eps = h->prm.omega = h->prm.g = h->prm.J_explicit = nullptr;
    h->prm.phonon_cap = nullptr;
    if (alloc && alloc->alloc && alloc->free) {
        h->alloc = *alloc;
        h->has_alloc = true;
    }
    h->st = (cudaStream_t)stream;

    // model tables
    DevModel* M = new DevModel();
    h->hmodel = M;
    s = paces::fill_model(params, L, M);
    if (s) {
        delete M;
        delete h;
        return s;
    }
    h->D = M->D;
    h->P = M->P;
    h->lpr = h->P <= 8 ? 1 : (h->P <= 24 ? 4 : 8);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete M;
        delete h;
        return PACES_ERR_CUDA;
    }
    Bufs& b = h->b;
    b.W = h->W;
    b.D = h->D;
    b.P = h->P;
    b.N = N;
    b.fmt = M->fmt;
    b.batch = h->R;
    b.G = std::min(kMaxChunkBlocks, h->sms * 4);
    b.grid = h->sms * 8;
    const int prec = prop_key(h);
    int bps = taylor_blocks_per_sm(h->lpr, prec);
    if (bps < 1) bps = 1;
    b.taylor_grid = h->sms * bps;
    int bps_max = std::max(std::max(taylor_blocks_per_sm(1, prec), taylor_blocks_per_sm(4, prec)),
                           taylor_blocks_per_sm(8, prec));
    b.rec_len = PACES_OBS_FIXED + 2 * N * h->R + (h->R > 1 ? 2 * h->R : 0);
    {   // bits each key word uses: the product of the radices packed into it
        unsigned __int128 prod[PACES_MAX_WORDS];
        for (int w = 0; w < PACES_MAX_WORDS; ++w) prod[w] = 1;
        prod[0] = h->lay.exciton_radix;
        for (int j = 0; j < N; ++j) prod[h->lay.site_word[j]] *= h->lay.site_radix[j];
        prod[h->lay.batch_word] *= h->lay.batch_radix;
        for (int w = 0; w < PACES_MAX_WORDS; ++w) {
            int bits = 0;
            while (w < h->W && bits < 64 && (((unsigned __int128)1) << bits) < prod[w]) ++bits;
            b.key_bits[w] = bits;
        }
    }

    b.model = alloc_track<DevModel>(h, h->fixed_allocs, 1);
    b.ctr = alloc_track<Counters>(h, h->fixed_allocs, 1);
    b.topq = alloc_track<TopqState>(h, h->fixed_allocs, 1);
    b.rs_hist = alloc_track<uint32_t>(h, h->fixed_allocs, 256 * (size_t)kMaxChunkBlocks + 256);
    b.blk_cnt = alloc_track<uint32_t>(h, h->fixed_allocs, kMaxChunkBlocks);
    b.blk_off = alloc_track<uint32_t>(h, h->fixed_allocs, kMaxChunkBlocks);
    b.partials = alloc_track<double>(h, h->fixed_allocs, 8 * (size_t)h->sms * std::max(bps, bps_max) + 16);
    b.obs_part = alloc_track<unsigned long long>(h, h->fixed_allocs,
                                                 std::max<size_t>((size_t)b.grid * (2 * kMaxSites + 1) * 2,
                                                                  (size_t)(2 * N * h->R + 1) * 2));
    if (h->R > 1) {      // per-realisation site energies for the diagonal
        double* e64 = alloc_track<double>(h, h->fixed_allocs, h->eps.size());
        dwf* edw = alloc_track<dwf>(h, h->fixed_allocs, h->eps.size());
        if (!e64 || !edw) {
            paces_destroy(h);
            return PACES_ERR_CAPACITY;
        }
        std::vector<dwf> hd(h->eps.size());
        for (size_t j = 0; j < hd.size(); ++j) hd[j] = dw_from_double(h->eps[j]);
        cudaMemcpyAsync(e64, h->eps.data(), h->eps.size() * 8, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(edw, hd.data(), hd.size() * sizeof(dwf), cudaMemcpyHostToDevice, h->st);
        cudaStreamSynchronize(h->st);
        M->eps_b64 = e64;
        M->eps_bdw = edw;
    }
    if (!b.model || !b.ctr || !b.blk_cnt || !b.blk_off || !b.partials || !b.obs_part ||
        cudaMallocHost(&h->hctr, sizeof(Counters)) != cudaSuccess) {
        paces_destroy(h);
        return PACES_ERR_CAPACITY;
    }
    std::memset(h->hctr, 0, sizeof(Counters));
    if (cudaMemcpyAsync((void*)b.model, M, sizeof(DevModel), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
        set_counters(h) != PACES_OK) {
        paces_destroy(h);
        return PACES_ERR_CUDA;
    }
    prepare_kernels(b);
    uint64_t want = params->max_rows ? params->max_rows : (uint64_t)kDefaultRows;
    if (grow(h, want, 0, 0) != PACES_OK) {
        paces_destroy(h);
        return PACES_ERR_CAPACITY;
    }
    *out = h;
    return PACES_OK;
}

paces_status paces_destroy(paces_t h)
{
    if (!h) return PACES_ERR_INVALID;
    cudaStreamSynchronize(h->st);
    drop_recording(h);
    free_rows(h);
    for (auto& a : h->fixed_allocs) dev_free(h, a);
    h->fixed_allocs.clear();
    cudaStreamSynchronize(h->st);
    for (auto e : h->evpool) cudaEventDestroy(e);
    invalidate_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->hctr) cudaFreeHost(h->hctr);
    delete h->hmodel;
    delete h;
    return PACES_OK;
}

const char* paces_last_error(paces_t h) { return h ? h->err.c_str() : "NULL handle"; }

// Encode n states in A form.  ncols = N: realisation 0 (replicated into every
// realisation of an ensemble when `replicate`); ncols = N + 1: the last column
// is the realisation.  Checks ranges and that no state repeats.
static paces_status encode_state(paces_t h, int64_t n, const int32_t* site, const int32_t* occ,
                                 std::vector<uint64_t>& keys, std::vector<uint32_t>& meta, int ncols,
                                 bool replicate, std::vector<int64_t>* src = nullptr)
{
    if (n <= 0 || !site || !occ) return fail(h, PACES_ERR_INVALID, "empty state or NULL arrays");
    const int N = h->N, W = h->W;
    int64_t copies = replicate ? h->R : 1;
    if ((uint64_t)n * copies > kMaxRowsHard) return fail(h, PACES_ERR_INVALID, "too many states");
    std::vector<int32_t> occN((size_t)n * N);
    std::vector<int32_t> real((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < N; ++j) {
            int32_t v = occ[i * ncols + j];
            if (v < 0 || v > h->cap[j]) return fail(h, PACES_ERR_INVALID, "occupation outside [0, phonon cap]");
            occN[i * N + j] = v;
        }
        if (ncols > N) {
            real[i] = occ[i * ncols + N];
            if (real[i] < 0 || real[i] >= h->R) return fail(h, PACES_ERR_INVALID, "realisation out of range");
        }
    }
    std::vector<uint64_t> base((size_t)n * W);
    std::string why;
    paces_status s = encode(&h->lay, n, site, occN.data(), base.data(), why);
    if (s) return fail(h, s, why);
    keys.resize((size_t)(n * copies) * W);
    meta.resize((size_t)(n * copies));
    if (src) src->resize((size_t)(n * copies));
    for (int64_t c = 0; c < copies; ++c)
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = c * n + i;
            for (int w = 0; w < W; ++w) keys[o * W + w] = base[i * W + w];
            uint64_t r = (uint64_t)(replicate ? c : real[i]);
            keys[o * W + h->lay.batch_word] += r * h->lay.batch_stride;
            int nph = 0;
            for (int j = 0; j < N; ++j) nph += occN[i * N + j];
            meta[o] = meta_pack(site[i], occN[i * N + site[i]], nph);
            if (src) (*src)[o] = i;
        }
    int64_t tot = n * copies;
    std::vector<int64_t> idx((size_t)tot);
    for (int64_t i = 0; i < tot; ++i) idx[i] = i;
    auto less = [&](int64_t a, int64_t b) {
        return std::lexicographical_compare(&keys[a * W], &keys[a * W] + W, &keys[b * W], &keys[b * W] + W);
    };
    std::sort(idx.begin(), idx.end(), less);
    for (int64_t i = 1; i < tot; ++i)
        if (std::equal(&keys[idx[i] * W], &keys[idx[i] * W] + W, &keys[idx[i - 1] * W]))
            return fail(h, PACES_ERR_INVALID, "duplicate basis states");
    return PACES_OK;
}

// Host amplitudes (re, im) in FP64 to the device storage format (16 bytes each).
static std::vector<float> to_dw(int64_t n, const double* amps)
{
    std::vector<float> out((size_t)n * 4);
    for (int64_t i = 0; i < 2 * n; ++i) {
        dwf d = dw_from_double(amps[i]);
        out[2 * i] = d.hi;
        out[2 * i + 1] = d.lo;
    }
    return out;
}

static paces_status upload_rows(paces_t h, int64_t n, const std::vector<uint64_t>& keys,
                                const std::vector<uint32_t>& meta, const double* amps, int vec)
{
    if ((uint64_t)n * 2 > h->cap_rows) {
        paces_status s = grow(h, (uint64_t)n * 2, 0, 0);
        if (s) return s;
    } else if (h->b.table_slots != (uint64_t)h->cap_rows * 100 / (uint64_t)h->table_pct + 1) {
        // a new table load: the same capacity with tables of the new size (the
        // state is replaced below, so nothing is kept)
        free_rows(h);
        Bufs nb = h->b;
        std::vector<DevAlloc> na;
        if (alloc_rows(h, h->cap_rows, na, nb) != PACES_OK) {
            h->has_state = false;
            h->cap_rows = 0;
            paces_status s = grow(h, (uint64_t)n * 2, 0, 0);
            if (s) return s;
        } else {
            h->row_allocs.swap(na);
            h->b = nb;
            invalidate_graphs(h);
        }
    }
    h->gen = 0;
    paces_status s = clear_table(h, 0);
    if (s) return s;
    CUDA_TRY(h, cudaMemcpyAsync(h->b.keys[0], keys.data(), keys.size() * 8, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(h->b.meta[0], meta.data(), meta.size() * 4, cudaMemcpyHostToDevice, h->st));
    if (h->b.fmt == 1) {
        CUDA_TRY(h, cudaMemcpyAsync(h->b.V[vec], amps, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice, h->st));
    } else {
        std::vector<float> d = to_dw(n, amps);
        CUDA_TRY(h, cudaMemcpyAsync(h->b.V[vec], d.data(), (size_t)n * 16, cudaMemcpyHostToDevice, h->st));
        CUDA_TRY(h, cudaStreamSynchronize(h->st));
    }
    count(h, Stage::Other, launch_insert_rows(h->b, 0, (uint32_t)n, h->st));
    std::memset(h->hctr, 0, sizeof(Counters));
    h->hctr->q = (uint32_t)n;
    h->hctr->q_in = (uint32_t)n;
    h->hctr->kept = (uint32_t)n;
    h->hctr->level_off[0] = 0;
    h->hctr->level_off[1] = (uint32_t)n;
    h->hctr->nlevels = 1;
    h->hctr->time = h->time;
    h->hctr->rec_index = h->n_records;
    CUDA_TRY(h, cudaMemsetAsync(h->b.obs_part, 0,
                                sizeof(unsigned long long) * 2 * std::max(2 * kMaxSites + 1, 2 * h->N * h->R + 1),
                                h->st));
    return set_counters(h);
}

paces_status paces_set_state(paces_t h, int64_t n, const int32_t* site, const int32_t* occ, const double* amps)
{
    if (!h) return PACES_ERR_INVALID;
    if (!amps) return fail(h, PACES_ERR_INVALID, "amps is NULL");
    std::vector<uint64_t> keys;
    std::vector<uint32_t> meta;
    std::vector<int64_t> src;
    paces_status s = encode_state(h, n, site, occ, keys, meta, h->N, true, &src);
    if (s) return s;
    std::vector<double> ramps(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        ramps[2 * i] = amps[2 * src[i]];
        ramps[2 * i + 1] = amps[2 * src[i] + 1];
    }
    amps = ramps.data();
    n = (int64_t)src.size();
    // psi(0) copy for the autocorrelation
    if (n > h->psi0_cap) {
        for (auto it = h->fixed_allocs.begin(); it != h->fixed_allocs.end();) {
            if (it->p == h->b.psi0_keys || it->p == h->b.psi0_amp) {
                dev_free(h, *it);
                it = h->fixed_allocs.erase(it);
            } else {
                ++it;
            }
        }
        h->b.psi0_keys = alloc_track<uint64_t>(h, h->fixed_allocs, (size_t)n * h->W);
        h->b.psi0_amp = alloc_track<double2>(h, h->fixed_allocs, (size_t)n);
        if (!h->b.psi0_keys || !h->b.psi0_amp) return fail(h, PACES_ERR_CAPACITY, "psi0 buffers");
        h->psi0_cap = n;
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->b.psi0_keys, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(h->b.psi0_amp, amps, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice, h->st));
    h->b.n0 = n;
    h->time = 0.0;
    h->n_records = 0;
    for (int attempt = 0;; ++attempt) {
        s = upload_rows(h, n, keys, meta, amps, 1);
        if (s) return s;
        int f = 0;
        bool overflow = false;
        for (; h->prm.m_init < 0 || f < h->prm.m_init; ++f) {
            count(h, Stage::Other, launch_level(h->b, 0, f, -1, -1, h->st));
            if (h->prm.m_init < 0 || f + 1 == h->prm.m_init) {
                s = read_counters(h);
                if (s) return s;
                if (h->hctr->err) {
                    overflow = h->hctr->err == kErrRows || h->hctr->err == kErrProbe || h->hctr->err == kErrCand;
                    if (!overflow) return fail(h, PACES_ERR_CUDA, "device error " + std::to_string(h->hctr->err));
                    break;
                }
                if (h->prm.m_init < 0 && h->hctr->level_off[f + 2] == h->hctr->level_off[f + 1]) break;
                if (f + 2 > kMaxLevels) return fail(h, PACES_ERR_UNSUPPORTED, "more than 256 BFS levels");
            }
        }
        CUDA_TRY(h, cudaGetLastError());
        if (!overflow) break;
        s = grow(h, (uint64_t)h->cap_rows + h->cap_rows / 8, 0, 0);
        if (s) return s;
    }
    h->fresh = true;
    h->has_state = true;
    h->csr_valid = false;
    h->last_truncated = false;
    h->time = 0.0;
    h->n_records = 0;
    s = ensure_obs(h, 1);
    if (s) return s;
    CUDA_TRY(h, cudaMemsetAsync(h->b.obs, 0, sizeof(double) * h->b.rec_len, h->st));
    count(h, Stage::Other, launch_observe(h->b, 0, h->b.V[1], 0.0, 1, h->st));
    s = read_counters(h);
    if (s) return s;
    if (h->hctr->err) return fail(h, PACES_ERR_CUDA, "device error " + std::to_string(h->hctr->err));
    h->n_records = 1;
    drop_recording(h);
    return PACES_OK;
}

paces_status paces_load_state(paces_t h, int64_t n, const int32_t* site, const int32_t* occ, const double* amps)
{
    if (!h) return PACES_ERR_INVALID;
    if (!amps) return fail(h, PACES_ERR_INVALID, "amps is NULL");
    std::vector<uint64_t> keys;
    std::vector<uint32_t> meta;
    paces_status s = encode_state(h, n, site, occ, keys, meta, h->N + (h->R > 1 ? 1 : 0), false);
    if (s) return s;
    s = upload_rows(h, n, keys, meta, amps, 0);
    if (s) return s;
    h->fresh = false;
    h->has_state = true;
    h->csr_valid = false;
    h->last_truncated = false;
    drop_recording(h);
    return PACES_OK;
}

// The step driver shared by threshold truncation (q_nom = 0) and top-q_nom
// truncation.
static paces_status step_impl(paces_t h, double dt, int64_t nsteps, double th2, int64_t q_nom, uint64_t seed)
{
    int64_t done = 0;
    std::vector<double> hrec;
    paces_status s = ensure_obs(h, h->n_records + nsteps);
    if (s) return s;
    bool recording = h->rec_every > 0 && h->rec_valid;
    while (done < nsteps) {
        int chunk = (int)std::min<int64_t>(kChunk, nsteps - done);
        if (recording) {
            if (h->rec_steps % h->rec_every == 0) {
                s = save_checkpoint(h);
                if (s) {
                    h->rec_valid = false;
                    return s;
                }
            }
            chunk = (int)std::min<int64_t>(chunk, h->rec_every - h->rec_steps % h->rec_every);
        }
        int g0 = h->gen;
        bool fresh0 = h->fresh;
        int64_t rec0 = h->n_records, step0 = h->step_index;
        for (int k = 0; k < chunk; ++k) enqueue_step(h, dt, th2, q_nom, seed, (size_t)k * 6);
        CUDA_TRY(h, cudaGetLastError());
        s = read_counters(h);
        if (s) return s;
        int err = h->hctr->err;
        // steps that completed wrote their record: the first missing one failed
        int64_t fs = (int64_t)h->hctr->rec_index - rec0;
        if (fs < 0 || fs > chunk) fs = 0;
        h->time = h->hctr->time;
        if (err == 0) {
            if (h->profiling) {
                hrec.resize((size_t)chunk * h->b.rec_len);
                CUDA_TRY(h, cudaMemcpy(hrec.data(), h->b.obs + rec0 * h->b.rec_len, sizeof(double) * hrec.size(),
                                       cudaMemcpyDeviceToHost));
                double prev_rows = 0.0;
                if (rec0 > 0)
                    CUDA_TRY(h, cudaMemcpy(&prev_rows, h->b.obs + (rec0 - 1) * h->b.rec_len + PACES_OBS_ROWS,
                                           sizeof(double), cudaMemcpyDeviceToHost));
                for (int k = 0; k < chunk; ++k) {
                    float ms;
                    for (int st = 0; st < 5; ++st)
                        if (cudaEventElapsedTime(&ms, ev(h, (size_t)k * 6 + st), ev(h, (size_t)k * 6 + st + 1)) ==
                            cudaSuccess)
                            h->stage_ms[st] += ms;
                    const double* r = hrec.data() + (size_t)k * h->b.rec_len;
                    double q_in = k == 0 ? prev_rows : hrec[(size_t)(k - 1) * h->b.rec_len + PACES_OBS_ROWS];
                    step_bytes(h, r, q_in, !(k == 0 && fresh0), h->stage_bytes);
                }
            }
            h->n_records += chunk;
            done += chunk;
            if (recording) {
                h->rec_steps += chunk;
                h->rec_dt.insert(h->rec_dt.end(), (size_t)chunk, dt);
                h->rec_th2.insert(h->rec_th2.end(), (size_t)chunk, th2);
                h->rec_nom.insert(h->rec_nom.end(), (size_t)chunk, q_nom);
                h->rec_seed.insert(h->rec_seed.end(), (size_t)chunk, seed);
            }
            continue;
        }
        // restore the host view at the start of the failed step
        int gen = g0;
        bool fresh = fresh0;
        for (int64_t k = 0; k < fs; ++k) {
            if (!fresh) gen = 1 - gen;
            fresh = false;
        }
        h->n_records = rec0 + fs;
        h->step_index = step0 + fs;
        done += fs;
        if (recording) {
            h->rec_steps += fs;
            h->rec_dt.insert(h->rec_dt.end(), (size_t)fs, dt);
            h->rec_th2.insert(h->rec_th2.end(), (size_t)fs, th2);
            h->rec_nom.insert(h->rec_nom.end(), (size_t)fs, q_nom);
            h->rec_seed.insert(h->rec_seed.end(), (size_t)fs, seed);
        }
        if (err == kErrRows || err == kErrProbe || err == kErrCand) {
            // the failing step's input (generation gen, vector V0) is intact
            uint32_t q = h->hctr->q_in;
            Counters keep = *h->hctr;
            h->gen = gen;
            h->fresh = fresh;
            std::memset(h->hctr, 0, sizeof(Counters));
            h->hctr->q = q;
            h->hctr->q_in = q;
            h->hctr->kept = q;
            h->hctr->level_off[1] = q;
            h->hctr->nlevels = 1;
            h->hctr->norm_last = keep.norm_last;
            h->hctr->time = keep.time;
            h->hctr->rec_index = keep.rec_index;
            s = set_counters(h);
            if (s) return s;
            s = grow(h, (uint64_t)h->cap_rows + h->cap_rows / 8, q, 0);
            if (s) return s;
            continue;
        }
        h->rec_valid = false;     // (capacity failures continued above)
        if (err == kErrNoConverge) {
            // the failed step's truncated and regrown state stays, unpropagated
            int nterm = h->hctr->err_info;
            h->gen = fresh ? gen : 1 - gen;
            h->fresh = true;
            h->csr_valid = false;
            h->hctr->err = 0;
            h->hctr->err_step = 0;
            s = set_counters(h);
            if (s) return s;
            return fail(h, PACES_ERR_NOCONVERGE,
                        std::string(h->prm.propagator == PACES_LANCZOS ? "Lanczos decomposition" : "Taylor series") +
                            " not converged after " + std::to_string(nterm) + " terms at step " +
                            std::to_string(h->step_index));
        }
        h->has_state = false;
        return fail(h, PACES_ERR_CUDA, "device error code " + std::to_string(err));
    }
    return PACES_OK;
}

paces_status paces_step(paces_t h, double dt, int64_t nsteps, double theta)
{
    if (!h) return PACES_ERR_INVALID;
    if (!(dt > 0.0) || nsteps < 0 || !(theta >= 0.0)) return fail(h, PACES_ERR_INVALID, "dt, nsteps or theta");
    if (!h->has_state) return fail(h, PACES_ERR_STATE, "no state: call paces_set_state first");
    return step_impl(h, dt, nsteps, theta * theta, 0, 0);
}

paces_status paces_step_nom(paces_t h, double dt, int64_t nsteps, int64_t q_nom, uint64_t seed)
{
    if (!h) return PACES_ERR_INVALID;
    if (!(dt > 0.0) || nsteps < 0 || q_nom < 1) return fail(h, PACES_ERR_INVALID, "dt, nsteps or q_nom");
    if (h->R > 1) return fail(h, PACES_ERR_UNSUPPORTED, "top-q_nom truncation covers batch 1 only");
    if (!h->has_state) return fail(h, PACES_ERR_STATE, "no state: call paces_set_state first");
    return step_impl(h, dt, nsteps, 0.0, q_nom, seed);
}

paces_status paces_set_coefficients(paces_t h, double J, const double* eps, const double* omega, const double* g)
{
    if (!h) return PACES_ERR_INVALID;
    if (h->rec_every > 0)
        return fail(h, PACES_ERR_UNSUPPORTED, "the reverse pass assumes one Hamiltonian for all recorded steps");
    const int N = h->N;
    std::vector<double> ne = h->eps, no = h->omega, ng = h->g;
    if (eps) ne.assign(eps, eps + (size_t)N * h->R);
    if (omega) no.assign(omega, omega + N);
    if (g) ng.assign(g, g + N);
    if (!std::isfinite(J)) return fail(h, PACES_ERR_INVALID, "J is not finite");
    for (double v : ne)
        if (!std::isfinite(v)) return fail(h, PACES_ERR_INVALID, "eps is not finite");
    for (int j = 0; j < N; ++j) {
        if (!std::isfinite(no[j]) || !std::isfinite(ng[j])) return fail(h, PACES_ERR_INVALID, "omega or g");
        if ((ng[j] == 0.0) != (h->g[j] == 0.0))
            return fail(h, PACES_ERR_INVALID, "g_s must stay zero exactly where it was (fixed move graph)");
    }
    if ((J == 0.0) != (h->prm.J == 0.0))
        return fail(h, PACES_ERR_INVALID, "J must stay zero exactly when it was (fixed move graph)");
    paces_params p = h->prm;
    p.J = J;
    p.eps = ne.data();
    p.omega = no.data();
    p.g = ng.data();
    p.phonon_cap = h->cap.data();
    p.J_explicit = h->Jx.empty() ? nullptr : h->Jx.data();
    DevModel* M = new DevModel();
    paces_status s = paces::fill_model(&p, h->lay, M);
    if (s) {
        delete M;
        return fail(h, s, "the new coefficients do not fit the model tables");
    }
    if (M->D != h->D || M->P != h->P) {
        delete M;
        return fail(h, PACES_ERR_INVALID, "the move graph changed");
    }
    M->eps_b64 = h->hmodel->eps_b64;        // ensembles: the device site-energy arrays stay
    M->eps_bdw = h->hmodel->eps_bdw;
    std::vector<dwf> hd;
    if (h->R > 1) {
        hd.resize(ne.size());
        for (size_t j = 0; j < hd.size(); ++j) hd[j] = dw_from_double(ne[j]);
        CUDA_TRY(h, cudaMemcpyAsync((void*)M->eps_b64, ne.data(), ne.size() * 8, cudaMemcpyHostToDevice, h->st));
        CUDA_TRY(h, cudaMemcpyAsync((void*)M->eps_bdw, hd.data(), hd.size() * sizeof(dwf), cudaMemcpyHostToDevice,
                                    h->st));
    }
    CUDA_TRY(h, cudaMemcpyAsync((void*)h->b.model, M, sizeof(DevModel), cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    delete h->hmodel;
    h->hmodel = M;
    h->prm.J = J;
    h->eps.swap(ne);
    h->omega.swap(no);
    h->g.swap(ng);
    return PACES_OK;
}

paces_status paces_num_rows(paces_t h, int64_t* rows)
{
    if (!h || !rows) return PACES_ERR_INVALID;
    paces_status s = read_counters(h);
    if (s) return s;
    *rows = h->has_state ? (int64_t)h->hctr->q : 0;
    return PACES_OK;
}

paces_status paces_get_state(paces_t h, int64_t max, int32_t* site, int32_t* occ, double* amps)
{
    if (!h) return PACES_ERR_INVALID;
    if (!h->has_state) return fail(h, PACES_ERR_STATE, "no state");
    paces_status s = read_counters(h);
    if (s) return s;
    uint32_t q = h->hctr->q;
    if (max < (int64_t)q) return fail(h, PACES_ERR_INVALID, "arrays smaller than the row count");
    if (q == 0) return PACES_OK;
    if (site || occ) {
        int32_t* ds = (int32_t*)dev_alloc(h, (size_t)q * 4);
        const int ncols = h->N + (h->R > 1 ? 1 : 0);
        int32_t* dox = (int32_t*)dev_alloc(h, (size_t)q * ncols * 4);
        if (!ds || !dox) return fail(h, PACES_ERR_CAPACITY, "export buffers");
        count(h, Stage::Other, launch_decode(h->b, h->gen, q, ds, dox, h->st));
        if (site) CUDA_TRY(h, cudaMemcpyAsync(site, ds, (size_t)q * 4, cudaMemcpyDeviceToHost, h->st));
        if (occ) CUDA_TRY(h, cudaMemcpyAsync(occ, dox, (size_t)q * ncols * 4, cudaMemcpyDeviceToHost, h->st));
        CUDA_TRY(h, cudaStreamSynchronize(h->st));
        dev_free(h, {ds, (size_t)q * 4});
        dev_free(h, {dox, (size_t)q * ncols * 4});
    }
    if (amps) {
        const double2* v = h->fresh ? h->b.V[1] : h->b.V[0];
        CUDA_TRY(h, cudaMemcpyAsync(amps, v, (size_t)q * sizeof(double2), cudaMemcpyDeviceToHost, h->st));
        CUDA_TRY(h, cudaStreamSynchronize(h->st));
        if (h->b.fmt == 0) {            // double-word pairs -> FP64, in place
            const float* f = reinterpret_cast<const float*>(amps);
            for (uint64_t i = 0; i < 2ull * q; ++i) {
                float hi = f[2 * i], lo = f[2 * i + 1];
                amps[i] = (double)hi + (double)lo;
            }
        }
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    return PACES_OK;
}

paces_status paces_get_levels(paces_t h, int64_t* off, int32_t max, int32_t* count_out)
{
    if (!h || !count_out) return PACES_ERR_INVALID;
    paces_status s = read_counters(h);
    if (s) return s;
    int32_t n = (int32_t)h->hctr->nlevels + 1;
    *count_out = n;
    for (int32_t i = 0; i < n && i < max && off; ++i) off[i] = h->hctr->level_off[i];
    return PACES_OK;
}

paces_status paces_get_keep(paces_t h, uint8_t* keep, int64_t max, int64_t* n)
{
    if (!h || !n) return PACES_ERR_INVALID;
    paces_status s = read_counters(h);
    if (s) return s;
    if (!h->last_truncated) {
        *n = 0;
        return PACES_OK;
    }
    uint32_t q = h->hctr->q_in;
    *n = q;
    if (!keep) return PACES_OK;
    if (max < (int64_t)q) return fail(h, PACES_ERR_INVALID, "keep array too small");
    std::vector<uint32_t> w(q / 32 + 1);
    CUDA_TRY(h, cudaMemcpyAsync(w.data(), h->b.keepw, w.size() * 4, cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    for (uint32_t i = 0; i < q; ++i) keep[i] = (w[i >> 5] >> (i & 31)) & 1u;
    return PACES_OK;
}

paces_status paces_get_hamiltonian(paces_t h, int32_t* cnt, int32_t* cols, double* vals, double* diag,
                                   int64_t max_nnz, int64_t* nnz)
{
    if (!h || !nnz) return PACES_ERR_INVALID;
    if (!h->has_state) return fail(h, PACES_ERR_STATE, "no state");
    if (!h->csr_valid) {
        CUDA_TRY(h, cudaMemsetAsync(&h->b.ctr->nnz, 0, 8, h->st));
        count(h, Stage::Other, launch_csr(h->b, h->gen, h->st));
        h->csr_valid = true;
    }
    paces_status s = read_counters(h);
    if (s) return s;
    uint32_t q = h->hctr->q;
    std::vector<uint8_t> c8(q);
    if (q) CUDA_TRY(h, cudaMemcpyAsync(c8.data(), h->b.cnt, q, cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    std::vector<uint64_t> off(q + 1, 0);
    for (uint32_t i = 0; i < q; ++i) off[i + 1] = off[i] + c8[i];
    *nnz = (int64_t)off[q];
    if (cnt)
        for (uint32_t i = 0; i < q; ++i) cnt[i] = c8[i];
    if (diag && q) {
        CUDA_TRY(h, cudaMemcpyAsync(diag, h->b.diag, (size_t)q * 8, cudaMemcpyDeviceToHost, h->st));
        CUDA_TRY(h, cudaStreamSynchronize(h->st));
        if (h->b.fmt == 0) {
            const float* f = reinterpret_cast<const float*>(diag);
            for (uint32_t i = 0; i < q; ++i) {
                float hi = f[2 * i], lo = f[2 * i + 1];
                diag[i] = (double)hi + (double)lo;
            }
        }
    }
    if ((cols || vals) && off[q] > 0) {
        if ((int64_t)off[q] > max_nnz) return fail(h, PACES_ERR_INVALID, "max_nnz too small");
        uint64_t* doff = (uint64_t*)dev_alloc(h, (size_t)q * 8);
        int32_t* dc = (int32_t*)dev_alloc(h, off[q] * 4);
        double* dv = (double*)dev_alloc(h, off[q] * 8);
        if (!doff || !dc || !dv) return fail(h, PACES_ERR_CAPACITY, "export buffers");
        CUDA_TRY(h, cudaMemcpyAsync(doff, off.data(), (size_t)q * 8, cudaMemcpyHostToDevice, h->st));
        count(h, Stage::Other, launch_export_csr(h->b, q, doff, dc, dv, h->st));
        if (cols) CUDA_TRY(h, cudaMemcpyAsync(cols, dc, off[q] * 4, cudaMemcpyDeviceToHost, h->st));
        if (vals) CUDA_TRY(h, cudaMemcpyAsync(vals, dv, off[q] * 8, cudaMemcpyDeviceToHost, h->st));
        CUDA_TRY(h, cudaStreamSynchronize(h->st));
        dev_free(h, {doff, (size_t)q * 8});
        dev_free(h, {dc, off[q] * 4});
        dev_free(h, {dv, off[q] * 8});
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    return PACES_OK;
}

paces_status paces_get_tuning(paces_t h, paces_tuning* out)
{
    if (!h || !out) return PACES_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    out->taylor_lanes_per_row = h->lpr;
    out->taylor_blocks_per_sm = h->b.taylor_grid / h->sms;
    out->grid_blocks_per_sm = h->b.grid / h->sms;
    out->chunk_blocks_per_sm = h->b.G / h->sms;
    out->use_graphs = h->use_graphs ? 1 : 0;
    out->max_taylor_blocks_per_sm = taylor_blocks_per_sm(h->lpr, prop_key(h));
    out->table_load_pct = h->table_pct;
    return PACES_OK;
}

paces_status paces_set_tuning(paces_t h, const paces_tuning* in)
{
    if (!h || !in) return PACES_ERR_INVALID;
    if (h->rec_steps > 0)
        return fail(h, PACES_ERR_STATE, "recorded steps must be replayed with the tuning they ran with");
    int lpr = in->taylor_lanes_per_row;
    if (lpr != 1 && lpr != 4 && lpr != 8) return fail(h, PACES_ERR_INVALID, "lanes per row must be 1, 4 or 8");
    int maxb = taylor_blocks_per_sm(lpr, prop_key(h));
    if (in->taylor_blocks_per_sm < 1 || in->taylor_blocks_per_sm > maxb)
        return fail(h, PACES_ERR_INVALID, "propagator blocks per SM must be 1.." + std::to_string(maxb));
    if (in->grid_blocks_per_sm < 1 || in->grid_blocks_per_sm > 32) return fail(h, PACES_ERR_INVALID, "grid blocks");
    if (in->chunk_blocks_per_sm < 1 || in->chunk_blocks_per_sm * h->sms > kMaxChunkBlocks)
        return fail(h, PACES_ERR_INVALID, "chunk blocks");
    if (in->table_load_pct != 0 && (in->table_load_pct < 20 || in->table_load_pct > 80))
        return fail(h, PACES_ERR_INVALID, "table load must be 20..80 percent");
    if (in->table_load_pct != 0) h->table_pct = in->table_load_pct;
    h->lpr = lpr;
    h->b.taylor_grid = h->sms * in->taylor_blocks_per_sm;
    h->b.grid = h->sms * in->grid_blocks_per_sm;
    h->b.G = h->sms * in->chunk_blocks_per_sm;
    h->use_graphs = in->use_graphs != 0;
    invalidate_graphs(h);
    return PACES_OK;
}

int32_t paces_record_len(paces_t h) { return h ? h->b.rec_len : 0; }

paces_status paces_selftest_barrier(int32_t extra_arrivals, double timeout_ms, int32_t* device_error)
{
    if (!device_error || extra_arrivals < 0 || !(timeout_ms > 0.0) || timeout_ms > 10000.0) return PACES_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return PACES_ERR_CUDA;
    Counters* ctr = nullptr;
    double* part = nullptr;
    const size_t pbytes = sizeof(double) * (4 * (size_t)sms + 8);
    if (cudaMalloc(&ctr, sizeof(Counters)) != cudaSuccess) return PACES_ERR_CUDA;
    if (cudaMalloc(&part, pbytes) != cudaSuccess) {
        cudaFree(ctr);
        return PACES_ERR_CUDA;
    }
    paces_status s = PACES_OK;
    Counters hc;
    if (cudaMemset(ctr, 0, sizeof(Counters)) != cudaSuccess || cudaMemset(part, 0, pbytes) != cudaSuccess ||
        launch_barrier_selftest(ctr, part, sms, (unsigned)(sms + extra_arrivals),
                                (unsigned long long)(timeout_ms * 1e6), 0) < 0 ||
        cudaStreamSynchronize(0) != cudaSuccess ||
        cudaMemcpy(&hc, ctr, sizeof(Counters), cudaMemcpyDeviceToHost) != cudaSuccess)
        s = PACES_ERR_CUDA;
    else
        *device_error = hc.err;
    cudaFree(part);
    cudaFree(ctr);
    return s;
}

paces_status paces_fp64_rate(double* tflops)
{
    if (!tflops) return PACES_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return PACES_ERR_CUDA;
    const int bps = fp64_rate_blocks_per_sm();
    if (bps < 1) return PACES_ERR_CUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PACES_ERR_CUDA;
    paces_status s = PACES_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        s = PACES_ERR_CUDA;
    } else {
        // one untimed launch, then the best of three timed ones
        for (int k = 0; k < 4 && s == PACES_OK; ++k) {
            float ms = 0.f;
            double fmas = 0.0;
            if (cudaEventRecord(e0, st) != cudaSuccess || (fmas = launch_fp64_rate(sms * bps, 2048, st)) < 0.0 ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
                s = PACES_ERR_CUDA;
                break;
            }
            if (k > 0) best = std::max(best, 2.0 * fmas / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (s == PACES_OK) *tflops = best;
    return s;
}

paces_status paces_num_records(paces_t h, int64_t* n)
{
    if (!h || !n) return PACES_ERR_INVALID;
    *n = h->n_records;
    return PACES_OK;
}

paces_status paces_observables(paces_t h, int64_t first, int64_t count_, double* out)
{
    if (!h || first < 0 || count_ < 0 || first + count_ > h->n_records || (count_ > 0 && !out))
        return fail(h, PACES_ERR_INVALID, "record range");
    if (count_ == 0) return PACES_OK;
    CUDA_TRY(h, cudaMemcpyAsync(out, h->b.obs + first * h->b.rec_len, sizeof(double) * h->b.rec_len * count_,
                                cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    return PACES_OK;
}

paces_status paces_profile(paces_t h, int32_t enable)
{
    if (!h) return PACES_ERR_INVALID;
    h->profiling = enable != 0;
    return PACES_OK;
}

paces_status paces_stage_stats(paces_t h, double* ms, int64_t* launches, double* bytes, int32_t reset)
{
    if (!h) return PACES_ERR_INVALID;
    for (int i = 0; i < PACES_NUM_STAGES; ++i) {
        if (ms) ms[i] = h->stage_ms[i];
        if (bytes) bytes[i] = h->stage_bytes[i];
    }
    for (int i = 0; i <= PACES_NUM_STAGES; ++i)
        if (launches) launches[i] = h->stage_launch[i];
    if (reset) {
        std::memset(h->stage_ms, 0, sizeof(h->stage_ms));
        std::memset(h->stage_bytes, 0, sizeof(h->stage_bytes));
        std::memset(h->stage_launch, 0, sizeof(h->stage_launch));
    }
    return PACES_OK;
}

paces_status paces_record(paces_t h, int32_t ckpt_every)
{
    if (!h || ckpt_every < 0) return PACES_ERR_INVALID;
    if (ckpt_every > 0 && h->R > 1) return fail(h, PACES_ERR_UNSUPPORTED, "the reverse pass covers batch 1 only");
    if (ckpt_every > 0 && h->prm.precision == PACES_C64_SPMV)
        return fail(h, PACES_ERR_UNSUPPORTED, "the reverse pass needs double-word or FP64 amplitudes");
    if (ckpt_every > 0 && h->prm.propagator == PACES_LANCZOS)
        return fail(h, PACES_ERR_UNSUPPORTED, "the reverse pass differentiates the Taylor propagator only");
    h->rec_every = ckpt_every;
    drop_recording(h);
    return PACES_OK;
}

paces_status paces_backward(paces_t h, int64_t nsteps, const double* dL_dc_final, const double* dL_dC,
                            const double* dL_dP, double* grad)
{
    if (!h || !grad) return PACES_ERR_INVALID;
    if (h->rec_every <= 0 || !h->rec_valid || !h->has_state)
        return fail(h, PACES_ERR_STATE, "no valid recording: call paces_record before stepping");
    if (nsteps <= 0 || nsteps != h->rec_steps)
        return fail(h, PACES_ERR_INVALID, "nsteps must equal the recorded steps (" + std::to_string(h->rec_steps) + ")");
    const int N = h->N, NP = 3 + N;
    const int64_t S = h->rec_every;
    const size_t rl = (size_t)h->b.rec_len;
    paces_status s = read_counters(h);
    if (s) return s;
    const Counters live_ctr = *h->hctr;
    const uint32_t q_live = live_ctr.q;
    const double live_time = h->time;

    // forward records of the recorded steps (restored unchanged at the end)
    std::vector<double> rec((size_t)nsteps * rl);
    CUDA_TRY(h, cudaMemcpyAsync(rec.data(), h->b.obs + (size_t)h->rec_base * rl, sizeof(double) * rec.size(),
                                cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    // a step of ns Taylor series with nt terms in all keeps nt + ns - 1 vectors
    // of its re-run: the terms of every series and the inputs of all but the first
    std::vector<uint32_t> qk((size_t)nsteps);
    std::vector<int> ntk((size_t)nsteps), nsk((size_t)nsteps);
    size_t term_bytes = 256, seg_bytes = 256;
    for (int64_t k = 0; k < nsteps; ++k) {
        qk[k] = (uint32_t)rec[(size_t)k * rl + PACES_OBS_ROWS];
        ntk[k] = (int)rec[(size_t)k * rl + PACES_OBS_TERMS];
        nsk[k] = std::max(1, (int)rec[(size_t)k * rl + PACES_OBS_SUBSTEPS]);
        term_bytes = std::max(term_bytes, (size_t)std::max(ntk[k] + nsk[k] - 1, 0) * qk[k] * 16);
    }
    if (qk[nsteps - 1] != q_live) return fail(h, PACES_ERR_STATE, "the live state is not the last recorded one");
    for (int64_t k0 = 0; k0 < nsteps; k0 += S) {
        size_t tot = 0, om, ov;
        for (int64_t k = k0 + 1; k < std::min(k0 + S, nsteps); ++k) tot += state_bytes(h, qk[k - 1], &om, &ov);
        seg_bytes = std::max(seg_bytes, tot);
    }

    // device scratch, released (and the live state restored) on every exit
    std::vector<DevAlloc> tmp;
    auto get = [&](size_t bytes) -> char* {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        void* p = dev_alloc(h, bytes);
        if (p) tmp.push_back({p, bytes});
        return (char*)p;
    };
    const uint64_t cap = h->cap_rows;
    size_t om, ov;
    char* live = get(state_bytes(h, q_live, &om, &ov));
    char* seg = get(seg_bytes);
    uint32_t* from = (uint32_t*)get(cap * 4);
    char* terms = get(term_bytes);
    double* acc = (double*)get(cap * 3 * 8);
    double2* G[2] = {(double2*)get(cap * 16), (double2*)get(cap * 16)};
    double2* MU[2] = {(double2*)get(cap * 16), (double2*)get(cap * 16)};
    unsigned long long* bins = (unsigned long long*)get((size_t)3 * NP * 8);
    double* dP = dL_dP ? (double*)get((size_t)nsteps * N * 8) : nullptr;
    double2* dC = dL_dC ? (double2*)get((size_t)nsteps * 16) : nullptr;
    bool ok = live && seg && from && terms && acc && G[0] && G[1] && MU[0] && MU[1] && bins &&
              (!dL_dP || dP) && (!dL_dC || dC);
    bool saved_live = false;
    auto finish = [&](paces_status st) -> paces_status {
        h->b.from = nullptr;
        h->b.terms = nullptr;
        h->b.term_max = 0;
        cudaGetLastError();
        std::string msg = h->err;
        if (saved_live) {
            paces_status r = restore_state(h, live, q_live, false, live_time, live_ctr.rec_index, &live_ctr);
            if (r == PACES_OK)
                r = cudaMemcpyAsync(h->b.obs + (size_t)h->rec_base * rl, rec.data(), sizeof(double) * rec.size(),
                                    cudaMemcpyHostToDevice, h->st) == cudaSuccess ? PACES_OK : PACES_ERR_CUDA;
            if (r != PACES_OK) {
                h->has_state = false;
                if (st == PACES_OK) st = r;
            }
            h->time = live_time;
        }
        cudaStreamSynchronize(h->st);
        for (auto& a : tmp) dev_free(h, a);
        cudaStreamSynchronize(h->st);
        h->csr_valid = false;
        h->last_truncated = false;
        if (st != PACES_OK && !msg.empty()) h->err = msg;
        return st;
    };
#define ADJ_TRY(call)                                                             \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return finish(cuda_fail(h, e_, #call));            \
    } while (0)
    if (!ok) return finish(fail(h, PACES_ERR_CAPACITY, "reverse-pass buffers"));
    s = copy_state_out(h, h->gen, 0, q_live, live);
    if (s) return finish(s);
    saved_live = true;

    ADJ_TRY(cudaMemsetAsync(bins, 0, (size_t)3 * NP * 8, h->st));
    if (dP) ADJ_TRY(cudaMemcpyAsync(dP, dL_dP, (size_t)nsteps * N * 8, cudaMemcpyHostToDevice, h->st));
    if (dC) ADJ_TRY(cudaMemcpyAsync(dC, dL_dC, (size_t)nsteps * 16, cudaMemcpyHostToDevice, h->st));
    int cur = 0;
    if (dL_dc_final)
        ADJ_TRY(cudaMemcpyAsync(G[cur], dL_dc_final, (size_t)q_live * 16, cudaMemcpyHostToDevice, h->st));
    else
        ADJ_TRY(cudaMemsetAsync(G[cur], 0, (size_t)q_live * 16, h->st));

    const int P = h->P;
    const int lpr = P <= 4 ? 1 : P <= 8 ? 2 : P <= 16 ? 4 : P <= 32 ? 8 : 16;
    std::vector<__int128> T((size_t)NP, 0);
    std::vector<unsigned long long> hb((size_t)3 * NP);
    int gen = 0;

    // one recorded step, replayed from the live buffers; capture: keep its
    // terms and row map for the reverse pass
    auto replay = [&](int64_t k, bool capture) -> paces_status {
        if (capture) {
            h->b.from = from;
            h->b.terms = terms;
            h->b.term_max = std::max(ntk[k] + nsk[k] - 1, 0);
        }
        gen = enqueue_kernels(h, h->st, h->gen, h->fresh, h->rec_dt[k], h->rec_th2[k], h->rec_nom[k], h->rec_seed[k],
                              (int)k, false, 0);
        h->gen = gen;
        h->b.from = nullptr;
        h->b.terms = nullptr;
        h->b.term_max = 0;
        CUDA_TRY(h, cudaGetLastError());
        paces_status r = read_counters(h);
        if (r) return r;
        if (h->hctr->err)
            return fail(h, PACES_ERR_CUDA, "device error " + std::to_string(h->hctr->err) + " replaying step " +
                                               std::to_string(k));
        if (h->hctr->q != qk[k] || (int)h->hctr->nterms != ntk[k] || h->hctr->nsub != nsk[k])
            return fail(h, PACES_ERR_STATE, "replay of recorded step " + std::to_string(k) + " diverged");
        h->fresh = false;
        return PACES_OK;
    };

    const int64_t nseg = (nsteps + S - 1) / S;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int64_t k0 = sg * S, k1 = std::min(k0 + S, nsteps);
        if (sg >= (int64_t)h->ckpts.size() || h->ckpts[sg].step != k0)
            return finish(fail(h, PACES_ERR_STATE, "missing checkpoint"));
        const paces_handle::Ckpt& C = h->ckpts[sg];
        // forward over the segment, keeping the input state of every step
        std::vector<size_t> off((size_t)(k1 - k0), 0);
        std::vector<double> tin((size_t)(k1 - k0), C.time);
        s = restore_state(h, (const char*)C.mem.p, C.q, C.fresh, C.time, h->rec_base + k0);
        if (s) return finish(s);
        size_t at = 0;
        for (int64_t k = k0; k + 1 < k1; ++k) {
            s = replay(k, false);
            if (s) return finish(s);
            off[k + 1 - k0] = at;
            tin[k + 1 - k0] = h->hctr->time;
            s = copy_state_out(h, gen, 0, qk[k], seg + at);
            if (s) return finish(s);
            at += state_bytes(h, qk[k], &om, &ov);
        }
        // reverse over the segment
        for (int64_t k = k1 - 1; k >= k0; --k) {
            if (k == k0) s = restore_state(h, (const char*)C.mem.p, C.q, C.fresh, C.time, h->rec_base + k0);
            else s = restore_state(h, seg + off[k - k0], qk[k - 1], false, tin[k - k0], h->rec_base + k);
            if (s) return finish(s);
            s = replay(k, true);
            if (s) return finish(s);
            const uint32_t q = qk[k];
            const int nt = ntk[k], ns = nsk[k];
            const double hs = h->rec_dt[k] / ns;
            double2* gb = G[cur];
            count(h, Stage::Other, launch_adj_obs(h->b, gen, h->b.V[0], dP ? dP + (size_t)k * N : nullptr,
                                                  dC ? dC + k : nullptr, gb, h->st));
            // stored vectors of the re-run: series 0 keeps phi_n at slot n - 1;
            // series j >= 1 keeps its input at slot b_j and phi_n at b_j + n
            std::vector<int> bj((size_t)ns, 0);
            for (int j = 1; j < ns; ++j) bj[j] = bj[j - 1] + h->hctr->sub_terms[j - 1] + (j > 1 ? 1 : 0);
            auto slot_ptr = [&](int sl) { return (const void*)(terms + (size_t)sl * q * 16); };
            const double2* mu = gb;
            int x = 0;
            bool first = true;
            for (int j = ns - 1; j >= 0; --j) {
                const int nj = h->hctr->sub_terms[j];
                for (int n = nj; n >= 1; --n) {
                    const void* phi;
                    if (j == 0) phi = n == 1 ? (const void*)h->b.V[1] : slot_ptr(n - 2);
                    else phi = slot_ptr(bj[j] + n - 1);
                    count(h, Stage::Other, launch_adj_term(h->b, lpr, mu, phi, gb, MU[x], acc, cap, hs / n, first,
                                                           h->st));
                    first = false;
                    mu = MU[x];
                    x ^= 1;
                }
                if (j > 0) {     // the input cotangent of series j is the output cotangent of series j-1
                    ADJ_TRY(cudaMemcpyAsync(gb, mu, (size_t)q * 16, cudaMemcpyDeviceToDevice, h->st));
                    mu = gb;
                }
            }
            if (nt >= 1) {
                count(h, Stage::Other, launch_adj_bins(h->b, gen, acc, cap, bins, h->st));
                ADJ_TRY(cudaMemcpyAsync(hb.data(), bins, hb.size() * 8, cudaMemcpyDeviceToHost, h->st));
                ADJ_TRY(cudaMemsetAsync(bins, 0, hb.size() * 8, h->st));
            }
            if (k > 0) {
                ADJ_TRY(cudaMemsetAsync(G[1 - cur], 0, (size_t)qk[k - 1] * 16, h->st));
                count(h, Stage::Other, launch_adj_scatter(h->b, from, mu, G[1 - cur], h->st));
            }
            ADJ_TRY(cudaGetLastError());
            s = read_counters(h);
            if (s) return finish(s);
            if (h->hctr->err == kErrGradRange)
                return finish(fail(h, PACES_ERR_INVALID, "a gradient contribution exceeds 2^50 in magnitude"));
            if (h->hctr->err) return finish(fail(h, PACES_ERR_CUDA, "device error " + std::to_string(h->hctr->err)));
            if (nt >= 1)
                for (int p = 0; p < NP; ++p) {
                    const __int128 two32 = (__int128)1 << 32, two64 = two32 * two32;
                    T[p] += (__int128)(int64_t)hb[3 * p + 2] * two64 + (__int128)hb[3 * p + 1] * two32 +
                            (__int128)hb[3 * p];
                }
            if (k > 0) cur ^= 1;
        }
    }
    for (int p = 0; p < NP; ++p) {
        int64_t hi = (int64_t)(T[p] >> 64);
        uint64_t lo = (uint64_t)(T[p] & (__int128)0xFFFFFFFFFFFFFFFFull);
        grad[p] = std::ldexp((double)hi, -8) + std::ldexp((double)lo, -72);
    }
    return finish(PACES_OK);
}
#undef ADJ_TRY

}  // extern "C"
