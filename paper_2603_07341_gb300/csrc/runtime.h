// runtime.h -- launch interface between the host runtime (paces_api.cu) and the
// kernel translation units.  Host-side declarations only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "paces.h"

namespace paces {

constexpr int kBlock = 256;        // threads of the chunked (scan-based) kernels
constexpr int kMaxChunkBlocks = 1024;

// Chunk [lo, hi) of n items owned by block b of G (multiples of kBlock), the
// split every scan-based kernel of one pass shares.
__device__ __forceinline__ void chunk_of(uint32_t n, uint32_t G, uint32_t b, uint32_t& lo, uint32_t& hi)
{
    uint32_t c = (n + G - 1) / G;
    c = (c + kBlock - 1) / kBlock * kBlock;
    uint64_t l = (uint64_t)b * c;
    lo = (uint32_t)(l < n ? l : n);
    uint64_t h = l + c;
    hi = (uint32_t)(h < n ? h : n);
}

// Selection state of top-q_nom truncation (kern_topq.cu).
struct TopqState {
    unsigned long long prefix;     // bits chosen so far in the current phase
    unsigned long long krem;       // rank still to place within the prefix
    unsigned long long w_cut;      // weight bits of the cut
    unsigned long long tk_cut;     // tie key of the cut (phase 1)
    uint32_t all;                  // q <= q_nom: every row is kept
    uint32_t phase;                // 0 weights, 1 tie keys, 2 done
    uint32_t ties_all;             // every row of the cut weight is kept
    uint32_t pad;
    uint32_t hist[4096];
};

// Device buffers of one handle (all device pointers).
struct Bufs {
    const DevModel* model;
    Counters* ctr;
    uint64_t* keys[2];             // row -> key, two generations
    uint32_t* meta[2];             // row -> (site, phonons at site, total phonons)
    uint64_t* table[2];            // hash tables, two generations
    uint64_t table_slots;          // slots per table (below 2^32)
    double2* V[4];                 // V0: state / accumulator r, V1: c' (phi_0), V2, V3: terms
    float2* F[2];                  // complex64 term buffers (C64_SPMV)
    uint32_t* col;                 // P H P columns, row pitch P
    uint8_t* cid;                  // coefficient ids, row pitch P
    uint8_t* cnt;                  // entries per row
    double* diag;                  // diagonal per row
    double* diag_h;                // FP64 propagator: h times the diagonal (h = dt / series)
    uint8_t* rperm;                // FP64 propagator: rows of each 256-row window by entry count
    uint32_t* cand_slot;           // candidate -> table slot, kCand | row (an existing row), or kNone
    uint32_t* from;                // adjoint re-runs: row -> row of the previous state (or kNone)
    uint64_t* sortk[2];            // sort of the kept set: keys (ping-pong)
    uint32_t* sorti[2];            // and their source rows
    uint32_t* rs_hist;             // digit counts per block [256][G]
    int key_bits[kMaxWords];       // bits used by each key word (radix passes)
    double2* kry;                  // Lanczos basis: kmax vectors of cap_rows rows
    void* terms;                   // adjoint re-runs: Taylor terms phi_1.. [n][row], 16 bytes each
    int term_max;                  // terms storable
    uint64_t* masks;               // winner bits per frontier row
    uint32_t* keepw;               // truncation bitmask
    uint32_t* blk_cnt;             // chunk counts
    uint32_t* blk_off;             // chunk offsets
    double* partials;              // Taylor reduction partials [2][G][4]
    TopqState* topq;               // top-q_nom selection state
    double* obs;                   // observables records
    unsigned long long* obs_part;  // observables partials [grid][2*kMaxSites+1][2]
    uint64_t* psi0_keys;
    double2* psi0_amp;
    int64_t n0;
    uint32_t cap_rows;
    uint64_t cand_cap;
    int W, D, P, N;
    int fmt;                        // amplitude storage: 0 double-word, 1 FP64
    int batch;                      // realisations of an ensemble (1: one model)
    int G;                          // blocks of chunked kernels
    int grid;                       // blocks of grid-stride kernels
    int taylor_grid;                // blocks of the cooperative propagator
    int rec_len;
};

struct TaylorParams {
    double dt;
    double xmax;                    // substeps: ceil(rho dt / xmax); <= 0: one series
    double tol2;
    int nmax;
    int fixed_terms;
    int step;
    int lpr;                        // lanes per row (1, 4 or 8)
    int c64;                        // complex64 SpMV terms
    int fmt;                        // amplitude storage: 0 double-word, 1 FP64
    int lanczos;                    // Lanczos decomposition (App. C.3) instead of the series
    int kmax;                       // Lanczos: most Krylov vectors per series
};

// Stage launchers; each returns the number of kernels it launched (or -1 on a
// launch error, which the caller reads with cudaGetLastError).
int launch_insert_rows(const Bufs& b, int gen, uint32_t n, cudaStream_t st);
int launch_truncate(const Bufs& b, int gin, int gout, double th2, int step, cudaStream_t st);
// Top-q_nom truncation: the selection writes the keep bits (kern_topq.cu), then
// the compaction shared with threshold truncation.
int launch_truncate_nom(const Bufs& b, int gin, int gout, uint64_t q_nom, uint64_t seed, int step,
                        cudaStream_t st);
int launch_topq_select(const Bufs& b, int gin, uint64_t q_nom, uint64_t seed, cudaStream_t st);
// The kept rows (keep bits and chunk offsets ready) compacted, sorted by key
// and placed in generation gout with their table (kern_sort.cu).
int launch_sorted_m(const Bufs& b, int gin, int gout, int step, cudaStream_t st);
int launch_level(const Bufs& b, int gen, int f, int rescue_gen, int step, cudaStream_t st);
int launch_csr(const Bufs& b, int gen, cudaStream_t st);
int launch_taylor(const Bufs& b, const TaylorParams& p, cudaStream_t st);
int launch_observe(const Bufs& b, int gen, const double2* vec, double dt, int mode, cudaStream_t st);
int prepare_kernels(const Bufs& b);
int launch_decode(const Bufs& b, int gen, uint32_t n, int32_t* site, int32_t* occ,
                  cudaStream_t st);
int launch_meta_from_keys(const Bufs& b, int gen, uint32_t n, cudaStream_t st);
int launch_export_csr(const Bufs& b, uint32_t q, const uint64_t* off, int32_t* cols,
                      double* vals, cudaStream_t st);

// Occupancy query key of the Lanczos propagator (precision values are 0..2).
constexpr int kPrecLanczos = 16;
int taylor_blocks_per_sm(int lpr, int precision);
double launch_fp64_rate(int grid, int iters, cudaStream_t st);
int fp64_rate_blocks_per_sm();
// Cooperative self-test of the bounded grid barrier (kern_taylor.cu).
int launch_barrier_selftest(Counters* ctr, double* part, int grid, unsigned expect, unsigned long long timeout_ns,
                            cudaStream_t st);

// Reverse pass of one step (kern_adjoint.cu).
int launch_adj_obs(const Bufs& b, int gen, const void* vec, const double* dLdP, const double2* wC, double2* gbar,
                   cudaStream_t st);
int launch_adj_term(const Bufs& b, int lpr, const double2* mu_in, const void* phi, const double2* gbar,
                    double2* mu_out, double* acc, uint64_t acc_stride, double s, int first, cudaStream_t st);
int launch_adj_bins(const Bufs& b, int gen, const double* acc, uint64_t acc_stride, unsigned long long* bins,
                    cudaStream_t st);
int launch_adj_scatter(const Bufs& b, const uint32_t* from, const double2* mu0, double2* gprev, cudaStream_t st);

// Host: plan the key layout and fill the device model description.
paces_status plan_layout_internal(const paces_params* params, paces_layout* out);
paces_status fill_model(const paces_params* params, const paces_layout& L, DevModel* M);

}  // namespace paces
