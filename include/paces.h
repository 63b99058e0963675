/*
 * paces.h -- C interface of the GB300 (sm_103a) per-timestep hot path of paces,
 * the co-evolving-subspace solver of the time-dependent Schroedinger equation
 * (arXiv 2603.07341).
 *
 * One handle evolves one single-exciton Holstein-type model (Eq. holstein):
 *
 *   H = sum_s eps_s |s><s| + J sum_{a != b} M_ab |a><b|
 *       + sum_j omega_j a_j^dag a_j + sum_s g_s |s><s| (a_s^dag + a_s),
 *
 * with a hard cap n_j <= K_j on the phonon number of site j (the paper's
 * d_pho - 1).  Time is in units of 1/omega_0 and hbar = 1.  A time step is the
 * map of Sec. 3.4, psi -> Q exp(-i P_m H P_m dt) psi, computed as
 *   (a1) truncation Q: keep the basis states whose weight |c|^2 reaches theta^2,
 *   (a2,a3) regrowth of H_eff to the ball of radius m around the kept set in the
 *        graph H induces on basis states (Eqs. def_neighbor, def_neighbor_k, H_eff),
 *        with de-duplication in a device hash table,
 *   (a4) rescue of amplitudes of states that were dropped and re-admitted
 *        ("post-adaptation detruncation", Sec. 3.3),
 *   (a5) the restricted Hamiltonian P_m H P_m as a sparse matrix (Sec. 3.3,
 *        "Generating the effective Hamiltonian"),
 *   (a6) the Taylor-series action of exp(-i P_m H P_m dt) by repeated SpMV (App. C.1),
 *   (a7) observables.
 *
 * Conventions, for every call below:
 *   - Host pointers are read during the call only; the library copies what it
 *     keeps.  The caller owns every array it passes.
 *   - The library owns its device memory.  It allocates through the allocator
 *     given to paces_create (or cudaMallocAsync when that is NULL), on the
 *     stream given to paces_create, and frees it in paces_destroy.
 *   - All device work is ordered on that stream.  Calls that return host data
 *     (paces_get_*, paces_observables) synchronise it.
 *   - Every call returns a status and never aborts the process.  After a
 *     failure, paces_last_error() describes it.  A failed paces_step leaves
 *     the state of the last completed step in place.
 *   - One handle must not be used from two threads at once.
 */
#ifndef PACES_H
#define PACES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paces_handle* paces_t;

typedef enum {
    PACES_OK = 0,
    PACES_ERR_INVALID = 1,     /* an argument is out of range or inconsistent      */
    PACES_ERR_KEY_WIDTH = 2,   /* the basis needs more than PACES_MAX_WORDS words  */
    PACES_ERR_CAPACITY = 3,    /* device memory ran out (after growing)            */
    PACES_ERR_NOCONVERGE = 4,  /* Taylor series not converged in taylor_nmax terms */
    PACES_ERR_CUDA = 5,        /* a CUDA runtime call failed                       */
    PACES_ERR_STATE = 6,       /* call out of order (e.g. step before set_state)   */
    PACES_ERR_UNSUPPORTED = 7  /* a size this build does not handle (see limits)   */
} paces_status;

/* build limits */
#define PACES_MAX_SITES 128     /* sites N                                   */
#define PACES_MAX_WORDS 4       /* 64-bit words per basis key (256 bits)     */
#define PACES_MAX_MOVES 64      /* off-diagonal moves per state (deg + 2)    */
#define PACES_MAX_COEFS 256     /* distinct off-diagonal matrix elements     */

/* lattice kinds: geometry that fixes the hopping pattern M_ab */
#define PACES_RING 0      /* 1D periodic: M = 1 on (j, j+1 mod N), pairs de-duplicated */
#define PACES_CHAIN 1     /* 1D open chain, site j at x = j (Eq. tb)                  */
#define PACES_OPEN2D 2    /* dims[0] x dims[1] open square lattice, j = x + dims0*y    */
#define PACES_OPEN3D 3    /* dims[0] x dims[1] x dims[2] open cubic lattice            */
#define PACES_EXPLICIT 4  /* M given in J_explicit[N*N] (symmetric, zero diagonal)    */
/* coupling kinds (geometric lattices): */
#define PACES_NEAREST 0   /* M_ab = 1 for Euclidean distance 1                         */
#define PACES_DIPOLAR 1   /* M_ab = 1 / r_ab^3 for all pairs (computed as 1/(r2*sqrt(r2))) */
/* arithmetic of the amplitudes and of the propagator */
#define PACES_C128 0      /* complex128: FP64 amplitudes and FP64 arithmetic, the         */
                          /* paper's (default)                                            */
#define PACES_DW 1        /* double-word: every amplitude is a pair of FP32 (48-bit       */
                          /* significand) and all arithmetic on them runs on the FP32     */
                          /* pipe with error-free transformations                         */
#define PACES_C64_SPMV 2  /* complex64 SpMV for the small terms of a series: from two     */
                          /* terms after the first whose norm is at most 2^-16 of the     */
                          /* state's (never before term 3); the leading terms, the        */
                          /* accumulator, norms and truncation magnitudes double-word     */

/* Device memory hook.  alloc returns device memory of `bytes` usable on
 * `stream` (a cudaStream_t) or NULL; free releases it.  Both may be called from
 * any paces_* call of the handle. */
typedef struct {
    void* ctx;
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} paces_allocator;

/* Model and method parameters (Eq. holstein; App. parameters for m, m_init). */
typedef struct {
    int32_t n_sites;            /* N, 1..PACES_MAX_SITES                                */
    int32_t lattice_kind;       /* PACES_RING .. PACES_EXPLICIT                         */
    int32_t dims[3];            /* lattice extents for OPEN2D / OPEN3D                  */
    int32_t coupling_kind;      /* PACES_NEAREST or PACES_DIPOLAR                       */
    double J;                   /* hopping scale: J_ab = J * M_ab                       */
    const double* J_explicit;   /* [N*N] pattern M for PACES_EXPLICIT, else NULL        */
    const double* eps;          /* [N] site energies eps_s, NULL = 0                    */
    const double* omega;        /* [N] phonon frequencies omega_j, NULL = 0             */
    const double* g;            /* [N] exciton-phonon couplings g_s, NULL = 0           */
    const int32_t* phonon_cap;  /* [N] K_j >= 0 (d_pho - 1), required                  */
    int32_t m;                  /* neighbour order of every step, >= 0 (paper: 2)       */
    int32_t m_init;             /* neighbour order of H_eff(0); < 0 = until closure     */
    int32_t precision;          /* PACES_C128, PACES_DW or PACES_C64_SPMV               */
    int32_t fixed_terms;        /* > 0: exactly this many series terms, no test         */
    double taylor_tol;          /* stop at n >= 2 with ||phi_n|| <= tol ||r||; 0 = 1e-15 */
    int32_t taylor_nmax;        /* series terms allowed before NOCONVERGE; 0 = 200      */
    uint64_t max_rows;          /* initial row capacity hint; 0 = automatic (it grows); */
                                /* at most 2^30 - 1 (paces_create: CAPACITY beyond)     */
    int32_t batch;              /* realisations R of a static-disorder ensemble (0 or 1 */
                                /* = one model); for R > 1 eps holds R*N site energies, */
                                /* realisation r in eps[r*N .. r*N + N)                 */
    int32_t reserved0;
    double taylor_xmax;         /* substepping (App. C.1): a step runs as               */
                                /* s = ceil(rho dt / xmax) Taylor series of dt / s,     */
                                /* rho = the largest absolute row sum of H over H_eff   */
                                /* (each term rounded up to 2^-20); 0 = 8; < 0 = always */
                                /* one series.  More than 1024 series: NOCONVERGE.      */
    int32_t propagator;         /* PACES_TAYLOR (0, default) or PACES_LANCZOS           */
    int32_t krylov_max;         /* PACES_LANCZOS: most Krylov vectors per series,       */
                                /* 1..PACES_MAX_KRYLOV; 0 = 30                          */
} paces_params;

/* Propagator of a6.  PACES_TAYLOR is the series of App. C.1.  PACES_LANCZOS is
 * the Lanczos decomposition App. C.3 compares it with:
 *   exp(-i h H) v ~ V_n exp(-i h T_n) V_n^dag v = ||v|| V_n exp(-i h T_n) e_1,
 * V_n the orthonormal Krylov basis of the three-term recurrence and T_n its
 * tridiagonal matrix, run over the same substeps h = dt / s.  A series stops at
 * the first n with h beta_n |(exp(-i h T_n) e_1)_n| <= taylor_tol (the norm of
 * the residual of the Krylov solution relative to ||v||, times h) and fails
 * with NOCONVERGE past krylov_max vectors.  It holds krylov_max vectors of 16
 * bytes per row of capacity on the device (the memory cost App. C.3 weighs
 * against the series) and applies H twice per vector's worth of streaming.
 * Requires PACES_C128 and batch <= 1, and cannot be recorded for the reverse
 * pass (paces_record: UNSUPPORTED).  The observables records' term count is the
 * number of Krylov vectors used. */
#define PACES_TAYLOR 0
#define PACES_LANCZOS 1
#define PACES_MAX_KRYLOV 32

/* Ensembles (batch = R > 1).  The R realisations share every parameter except
 * the site energies.  They are evolved together as one block-diagonal problem:
 * the realisation index r is one more digit of every basis key, which no move
 * changes, so one H_eff, one hash table and one launch of every stage serve all
 * realisations, whatever their subspace sizes.  paces_set_state replicates
 * psi(0) into every realisation; paces_get_state and paces_load_state carry r
 * as an extra last column of occ (N + 1 columns).  Rows of one realisation
 * appear in the same relative order as in a run of that realisation alone.
 * The Taylor series stops on the norms of the whole ensemble.  Observables
 * records then hold, after the fixed fields, P_s for every (r, s), <n_j> for
 * every (r, j) and C_r(t) (re, im) for every r; the fixed C field is the mean
 * over r.  Limit: R <= PACES_MAX_BATCH. */
#define PACES_MAX_BATCH 4096

/* Basis-key layout (App. A, generalised to mixed radix): a state (s, n_0..n_{N-1})
 * is the integer  s + N_s * sum_j n_j R_j  split over `words` 64-bit words; no
 * digit straddles a word.  Word 0 holds the exciton digit s (radix exciton_radix)
 * in its lowest position; site j lives in word site_word[j] with place value
 * site_stride[j] and radix site_radix[j] (K_j + 1, or the next power of two when
 * pow2 != 0, which is chosen whenever it needs no more words).  The all-ones key
 * is never a valid state. */
typedef struct {
    int32_t n_sites;
    int32_t words;
    int32_t pow2;
    int32_t reserved;
    uint64_t exciton_radix;
    int32_t site_word[PACES_MAX_SITES];
    uint64_t site_stride[PACES_MAX_SITES];
    uint64_t site_radix[PACES_MAX_SITES];
    int32_t batch_word;         /* ensembles: word, place value and radix of the   */
    int32_t reserved1;          /* realisation digit (radix 1 for a single model)  */
    uint64_t batch_stride;
    uint64_t batch_radix;
} paces_layout;

/* Host-only: plan the key layout of a model.  No GPU is touched.
 * Returns INVALID for bad parameters, KEY_WIDTH if the basis needs more than
 * PACES_MAX_WORDS words. */
paces_status paces_plan_layout(const paces_params* params, paces_layout* out);

/* Host-only: encode n states given in A form (App. A: site[n], occ[n*N]) into
 * keys[n*words] (word 0 first), in realisation 0 of an ensemble.  Returns
 * INVALID if a digit is out of range. */
paces_status paces_encode_keys(const paces_layout* layout, int64_t n, const int32_t* site,
                               const int32_t* occ, uint64_t* keys);

/* Create a handle.  params is copied.  alloc may be NULL (cudaMallocAsync).
 * stream is a cudaStream_t (NULL = legacy default stream).  The current CUDA
 * device at this call is the handle's device.  Returns INVALID, KEY_WIDTH,
 * UNSUPPORTED (more than PACES_MAX_MOVES moves or PACES_MAX_COEFS distinct
 * matrix elements), CAPACITY or CUDA. */
paces_status paces_create(const paces_params* params, const paces_allocator* alloc,
                          void* stream, paces_t* out);

/* Release all device memory of the handle (stream-ordered) and the handle. */
paces_status paces_destroy(paces_t h);

/* Text of the last error of the handle ("" if none); valid until the next call. */
const char* paces_last_error(paces_t h);

/* Set psi(0) (Sec. 2; input in A form, App. A): n > 0 distinct states site[n],
 * occ[n*N], amplitudes amps[2n] as (re, im).  H_eff(0) becomes the ball of
 * radius m_init around them (Eq. H_eff with m = m_init); the first paces_step
 * propagates in it without truncating.  psi(0) is also the reference of the
 * autocorrelation C(t) = <psi(0)|psi(t)> (Sec. 5, Eq. init_state_spec).
 * Clears the observables.  Returns INVALID (duplicates, digits out of range),
 * CAPACITY or CUDA. */
paces_status paces_set_state(paces_t h, int64_t n, const int32_t* site, const int32_t* occ,
                             const double* amps);

/* Load a mid-trajectory state: n distinct rows with amplitudes become the
 * current H_eff and vector exactly as a completed step leaves them, so the next
 * paces_step truncates and regrows from it.  The C(t) reference is kept
 * (C = 0 if paces_set_state was never called).  Observables are kept. */
paces_status paces_load_state(paces_t h, int64_t n, const int32_t* site, const int32_t* occ,
                              const double* amps);

/* Advance nsteps time steps of length dt (> 0) with amplitude threshold theta
 * (>= 0): keep a row iff re^2 + im^2 >= theta^2 (PACES_C128: in FP64 without
 * contraction; double-word storage: in double-word arithmetic, relative error
 * below 2^-46).  Row order after a step: the kept set M in ascending basis
 * order (n_{N-1} most significant, down to n_0, then s; the realisation first
 * in an ensemble), then each regrown BFS level in first-occurrence order
 * (parents in row order, moves in canonical order).  Appends one observables
 * record per step.  Capacity grows automatically (up to 2^30 - 1 rows) and the
 * failing step is redone.  Returns INVALID, STATE (no
 * state set), NOCONVERGE (series did not reach taylor_tol: the state stays as
 * the failed step truncated and regrew it, unpropagated, and the next call
 * propagates it without truncating again), CAPACITY or CUDA. */
paces_status paces_step(paces_t h, double dt, int64_t nsteps, double theta);

/* As paces_step, with the paper's own truncation (Sec. "Truncation &
 * post-adaptation detruncation"; App. "How to weight states for truncation"):
 * keep the q_nom (>= 1) rows of largest weight w = re^2 + im^2 (all rows when
 * q <= q_nom), then regrow and rescue as usual, so H_eff has q_true >= q_nom
 * rows.  w is compared as FP64 (PACES_C128: products and sum rounded
 * separately; double-word storage: the double-word |c|^2 rounded to FP64).
 * Degenerate weights at the cutoff are ordered by
 *   tk = (u & 0xFFFFFFFF00000000) | (0xFFFFFFFF - row),
 * u = the hash of (seed, t, s, n_0 .. n_{N-1}): z = seed + G t, then
 * z = mix(z ^ v) for each entry v in that order, with mix the SplitMix64
 * output function (Steele, Lea & Flood 2014), G = 0x9E3779B97F4A7C15 and t
 * the index of the observables record the step writes (1 for the first step
 * after paces_set_state); larger (w, tk) is kept first, so exactly q_nom rows
 * are kept when q > q_nom.  The selection runs on the device (radix select of
 * the weight bits, then of the tie keys of the rows at the cut weight).  The
 * record's KEPT field holds |M| and ROWS holds q_true.  Returns as paces_step,
 * and UNSUPPORTED for ensembles (batch > 1). */
paces_status paces_step_nom(paces_t h, double dt, int64_t nsteps, int64_t q_nom, uint64_t seed);

/* Time-dependent Hamiltonians that are piecewise constant in time (the
 * extension Sec. 6 describes: the Hamiltonian is adjusted at every time step,
 * with its coupling magnitudes changing and its graph fixed).  Replaces, for
 * the steps that follow, the hopping scale J (J_ab = J M_ab with the pattern M
 * of paces_create), and, where the pointer is not NULL, eps[N] (or eps[R*N]
 * for an ensemble), omega[N] and g[N] (copied).  The move graph may not
 * change: J must be zero exactly when it was, and each g_s zero exactly where
 * it was (INVALID otherwise).  Stream-ordered before the next step; the steps
 * already taken are unaffected.  UNSUPPORTED while paces_record is on (the
 * reverse pass assumes one Hamiltonian for all recorded steps); CAPACITY if
 * the new values have more distinct off-diagonal elements than
 * PACES_MAX_COEFS. */
paces_status paces_set_coefficients(paces_t h, double J, const double* eps, const double* omega,
                                    const double* g);

/* Number of rows q = dim H_eff of the current state. */
paces_status paces_num_rows(paces_t h, int64_t* rows);

/* Copy the current state to the host in row order: site[rows], occ[rows*N],
 * amps[2*rows].  max is the capacity of the arrays in rows; INVALID if smaller
 * than the row count.  Any pointer may be NULL to skip that array. */
paces_status paces_get_state(paces_t h, int64_t max, int32_t* site, int32_t* occ,
                             double* amps);

/* Row offsets of the BFS levels of the current H_eff: level 0 (the kept set M,
 * or psi(0)) is rows [off[0], off[1]), level k rows [off[k], off[k+1]).
 * Writes up to max entries and the count (levels + 1) to *count. */
paces_status paces_get_levels(paces_t h, int64_t* off, int32_t max, int32_t* count);

/* Truncation mask of the last step over the rows that entered it (1 = kept).
 * *n receives its length (0 when the last step did not truncate). */
paces_status paces_get_keep(paces_t h, uint8_t* keep, int64_t max, int64_t* n);

/* The restricted Hamiltonian P_m H P_m of the current H_eff as the kernels hold
 * it: per row the count cnt[rows] of off-diagonal entries, their columns and
 * values in move order (cols/vals of length max_nnz, rows back to back), and
 * the diagonal diag[rows].  *nnz receives the off-diagonal total; INVALID if it
 * exceeds max_nnz.  Pointers may be NULL (then only *nnz is returned). */
paces_status paces_get_hamiltonian(paces_t h, int32_t* cnt, int32_t* cols, double* vals,
                                   double* diag, int64_t max_nnz, int64_t* nnz);

/* Observables, one record per time index (0 = psi(0), k = after step k).
 * Each record has paces_record_len() doubles: the fields below, then the site
 * populations P_s (N values; Eq. RMSD uses them) and the mean phonon numbers
 * <n_j> (N values); for ensembles see PACES_MAX_BATCH above. */
#define PACES_OBS_TIME 0         /* t                                           */
#define PACES_OBS_NORM 1         /* ||c||^2 after the step                      */
#define PACES_OBS_NORM_PHI0 2    /* ||c'||^2 entering the propagator            */
#define PACES_OBS_ENERGY 3       /* <c'|P H P|c'>                               */
#define PACES_OBS_C_RE 4         /* C(t) = <psi(0)|psi(t)>, real part            */
#define PACES_OBS_C_IM 5
#define PACES_OBS_ROWS 6         /* q = dim H_eff                               */
#define PACES_OBS_KEPT 7         /* |M| after truncation                        */
#define PACES_OBS_NNZ 8          /* stored entries of P H P incl. the diagonal  */
#define PACES_OBS_TERMS 9        /* Taylor terms (Lanczos: Krylov vectors) used  */
#define PACES_OBS_NORM_BEFORE 10 /* ||c||^2 before truncation                   */
#define PACES_OBS_SUBSTEPS 11    /* Taylor series the step ran (substeps)       */
#define PACES_OBS_HBOUND 12      /* rho, the bound on ||P H P|| that set them    */
#define PACES_OBS_FIXED 14       /* fields before P_s                           */
int32_t paces_record_len(paces_t h);
/* Number of records held. */
paces_status paces_num_records(paces_t h, int64_t* n);
/* Copy records [first, first + count) to out[count * record_len]. */
paces_status paces_observables(paces_t h, int64_t first, int64_t count, double* out);

/* Stage timing (CUDA events on the handle's stream) and launch counting.
 * Stages: 0 truncation, 1 expansion+dedup+rescue, 2 Hamiltonian build,
 * 3 propagation, 4 observables. */
#define PACES_NUM_STAGES 5
paces_status paces_profile(paces_t h, int32_t enable);
/* ms[5]: summed stage times since the last reset; launches[6]: kernels launched
 * per stage (index 5: set_state and other kernels); bytes[5]: algorithmic bytes
 * moved per stage: per row, the key and amplitude reads and writes each stage
 * must make, one 32-byte sector per hash probe, 5 bytes per stored entry of
 * P H P, and per Taylor term 1 + 8 + 16 + 16 + 32 bytes per row. */
paces_status paces_stage_stats(paces_t h, double* ms, int64_t* launches, double* bytes,
                               int32_t reset);

/* Launch shapes and step replay (no counterpart in the paper).  Read the
 * current values, change some and write them back; the project autotuner
 * (paper_2603_07341_gb300/autotune.py) picks them by timing steps.  Results do
 * not depend on them except through the summation order of reductions.
 * Returns INVALID for out-of-range values. */
typedef struct {
    int32_t taylor_lanes_per_row;     /* 1, 4 or 8 lanes per row of P H P in the propagator  */
    int32_t taylor_blocks_per_sm;     /* cooperative 256-thread blocks per SM, 1..max below   */
    int32_t grid_blocks_per_sm;       /* blocks per SM of the grid-stride kernels, 1..32      */
    int32_t chunk_blocks_per_sm;      /* blocks per SM of the scan-based kernels (total <= 1024) */
    int32_t use_graphs;               /* 1: every step is captured once as a CUDA graph and   */
                                      /* replayed (not while stage timing is on)              */
    int32_t max_taylor_blocks_per_sm; /* read only: co-residency limit of the propagator      */
    int32_t table_load_pct;           /* largest load of the hash tables in percent, 20..80   */
                                      /* (slots = rows of capacity x 100 / pct + 1; default   */
                                      /* 50); 0 keeps it.  Takes effect when the tables are   */
                                      /* next allocated: the next paces_set_state or          */
                                      /* paces_load_state, or capacity growth.  CAPACITY when */
                                      /* a table would need 2^31 slots or more.               */
    int32_t reserved;
} paces_tuning;
paces_status paces_get_tuning(paces_t h, paces_tuning* out);
paces_status paces_set_tuning(paces_t h, const paces_tuning* in);

/* ---- Gradients (an extension: the paper defines the forward map only) -----
 * Reverse-mode derivative of a loss of recorded steps with respect to the
 * model parameters p = [J, g, omega, eps_0 .. eps_{N-1}] of Eq. holstein:
 * J scales every hopping amplitude (J_ab = J M_ab), g scales every g_j,
 * omega shifts every omega_j together, eps_s is the energy of exciton site s.
 * The subspace sequence (truncation Q, regrowth, rescue; Sec. 3) and the
 * number of Taylor terms of every step (Eq. taylor) are held at the values the
 * forward steps took: the derivative is that of the recorded map, which is
 * what central differences with the truncation masks held fixed measure.
 *
 * paces_record(h, k): from the current state on (or from the next set_state
 * or load_state), keep a copy of the state every k recorded steps (keys, row
 * descriptors and amplitudes; about 8W + 20 bytes per row) plus dt and theta
 * of every step.  k = 0 stops recording and frees the copies.  A new state
 * restarts the recording.  UNSUPPORTED for batch > 1 or PACES_C64_SPMV.  While
 * steps are recorded paces_set_tuning returns STATE (the replay must repeat
 * the forward's reduction order bit for bit).  A step that fails for any
 * reason other than capacity ends the recording (backward then returns STATE).
 *
 * paces_backward(h, nsteps, dL_dc_final, dL_dC, dL_dP, grad): nsteps must be
 * the number of recorded steps.  Cotangents (host arrays, each may be NULL):
 *   dL_dc_final [2 q]       dL/dRe c + i dL/dIm c on the rows of the current
 *                           state, in paces_get_state order (re, im pairs);
 *   dL_dC       [2 nsteps]  dL/dRe C + i dL/dIm C of the autocorrelation
 *                           C(t) = <psi(0)|psi(t)> after recorded step k;
 *   dL_dP       [nsteps N]  dL/dP_s of the site populations after step k.
 * grad [3 + N] receives dL/dp.  The pass replays each segment of k steps from
 * its copy, then re-runs every step once more keeping its Taylor terms
 * (16 bytes per row per term) and its row map, and runs the reverse
 * recurrence mu_{n-1} = gbar + (i dt / n) H mu_n in FP64.  Gradient sums are
 * exact fixed-point integers (2^-72), independent of thread timing.  The
 * current state and the observable records are restored unchanged; the
 * recording stays valid.  Errors: STATE (no valid recording, or a replayed
 * step diverged from its record), INVALID (nsteps, NULL grad, a per-row
 * contribution beyond 2^50), CAPACITY (scratch of about 100 bytes per row of
 * capacity plus the terms of the largest step). */
paces_status paces_record(paces_t h, int32_t ckpt_every);
paces_status paces_backward(paces_t h, int64_t nsteps, const double* dL_dc_final, const double* dL_dC,
                            const double* dL_dP, double* grad);

/* ---- Self-test of the bounded grid barrier (no counterpart in the paper) ----
 * The propagator runs all Taylor terms of a step in one cooperative launch
 * whose blocks meet at a grid barrier after every term; every wait there is
 * bounded, and a wait that runs out records a device error instead of hanging.
 * This call exercises that path on the current device: one 256-thread block
 * per SM arrives at a barrier that expects (SMs + extra_arrivals) arrivals,
 * with a limit of timeout_ms (0 < timeout_ms <= 10000).  extra_arrivals = 0:
 * the barrier completes and *device_error = 0; extra_arrivals > 0: no block is
 * the last to arrive, every wait runs out and *device_error = 5 (the barrier
 * error code).  The context stays usable.  Allocates and frees its own small
 * buffers with cudaMalloc.  Returns INVALID or CUDA. */
paces_status paces_selftest_barrier(int32_t extra_arrivals, double timeout_ms, int32_t* device_error);

/* ---- FP64 rate probe (no counterpart in the paper) -------------------------
 * The complex128 propagator is bound by the FP64 pipe, so its roofline needs
 * the FP64 rate the GPU actually sustains next to the one derived from unit
 * counts and clocks.  On the current device this runs a kernel whose threads
 * (as many as fit on every SM) each keep eight independent FP64 FMA chains
 * going, once untimed and three times timed with CUDA events on a stream of
 * its own, and stores the best rate in *tflops (TFLOP/s, two flops per FMA).
 * Synchronises that stream; allocates no device memory.  Returns INVALID
 * (tflops NULL) or CUDA. */
paces_status paces_fp64_rate(double* tflops);

/* ---- Expansion without allocation (no counterpart in the paper) -----------
 * Some callers cannot allocate device memory: hosts whose framework has
 * already reserved all of it in its own pool, real-time loops that must never
 * enter an allocator, or code running under a policy that forbids a library
 * from allocating.  For them this call performs one level of the expansion
 * (a2/a3 above) with all of its working memory -- model tables, counters, the
 * hash table, candidate slots and winner masks -- in one fixed device array of
 * PACES_NOALLOC_SCRATCH_BYTES that the library reserves on every GPU that
 * loads it and holds until the process exits.  It calls no cudaMalloc,
 * cudaMallocAsync, cudaFree or allocating library routine.
 *
 * keys_in:  device array of n_in >= 1 distinct keys (paces_encode_keys
 *           layout, words per key from paces_plan_layout), not modified.
 * keys_out: device array of max_out keys (max_out >= n_in), caller-owned.
 *           Receives the input keys in order, then every state reachable by
 *           one move of H and not among them, in first-occurrence order
 *           (inputs in order, moves in canonical order) -- exactly the rows
 *           paces_set_state produces with m_init = 1.  *n_out gets the count.
 * stream:   a cudaStream_t; the call synchronises it before returning.
 *
 * Limit: every piece of working memory must fit in the array, i.e.
 *   68 KB (model tables and counters) + 8 KB (chunk counts)
 *   + (2 R + 1) * 8 * S  (hash table; S = 2, 4, 4, 6 words for 1..4 key words)
 *   + n_in * (4 D + 8) + 20 R bytes,
 * with R = min(max_out, n_in (D + 1)) and D = max moves per state (the
 * largest number of hops from a site, plus 2).  Larger requests, and outputs
 * that would exceed max_out, return PACES_ERR_CAPACITY and leave keys_out
 * undefined; INVALID, KEY_WIDTH or UNSUPPORTED are returned as by
 * paces_create.
 *
 * The array is shared by every call in the process and keeps the previous
 * call's contents; each call re-initialises what it reads.  Calls whose GPU
 * work overlaps (two threads, or two streams of one thread) race on it and
 * must be serialised by the caller.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it; make that first call before any stream capture. */
#define PACES_NOALLOC_SCRATCH_BYTES (32u << 20)
paces_status paces_expand_noalloc(const paces_params* params, const uint64_t* keys_in, int64_t n_in,
                                  uint64_t* keys_out, int64_t max_out, int64_t* n_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
