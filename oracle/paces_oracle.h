/*
 * paces_oracle.h -- interface of the plain CPU oracle of the co-evolving-subspace
 * time step (Sec. 3.4 of the paces paper, arXiv 2603.07341).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is loaded by the test suite, by the
 * package's smoke check and by the benchmark's CPU-baseline leg.  The product
 * path (the CUDA library and its Python binding) never loads, calls or links it,
 * and the oracle shares no code, header, table or helper with that path.
 *
 * Everything is FP64, single-threaded, and written for legibility, not speed.
 * Basis states are plain integer tuples (s, n_0, ..., n_{N-1}): exciton site s
 * and one phonon occupation per site (Eq. holstein).
 */
#ifndef PACES_ORACLE_H
#define PACES_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle oracle_t;

/* status codes (same meaning as the product's, numbered independently) */
#define OR_OK 0
#define OR_INVALID 1
#define OR_NOMEM 3
#define OR_NOCONVERGE 4
#define OR_STATE 6

/* lattice kinds: 0 ring, 1 open chain, 2 open 2D, 3 open 3D, 4 explicit matrix
 * coupling kinds: 0 nearest neighbour (distance 1), 1 all pairs J / r^3      */
oracle_t* or_create(int n_sites, int lattice_kind, const int* dims, int coupling_kind,
                    double J, const double* J_explicit, const double* eps,
                    const double* omega, const double* g, const int* cap,
                    int m, int m_init, double tol, int nmax, int fixed_terms);
void or_destroy(oracle_t* o);

/* Substepping (App. C.1, the scaling alternative to one series per step): a
 * step of length dt runs as s = ceil(rho dt / xmax) series of length dt / s,
 * rho the largest absolute row sum of H over the rows of H_eff (see
 * paces_oracle.c).  xmax <= 0: always one series.  Default 8. */
int or_set_xmax(oracle_t* o, double xmax);

/* Propagator of a step: kind 0 the Taylor series of App. C.1 (default), kind 1
 * the Lanczos decomposition of App. C.3 with at most kmax Krylov vectors per
 * series (1 <= kmax <= OR_MAX_KRYLOV); the same substep split applies to both.
 * Lanczos steps cannot be recorded for the adjoint (OR_INVALID). */
#define OR_MAX_KRYLOV 64
int or_set_propagator(oracle_t* o, int kind, int kmax);
/* Orthonormal Lanczos vectors v_1..v_n of the last series of the last Lanczos
 * step: fills V[2*q*k + 2*i + {0,1}] (re, im of row i of v_{k+1}) for k <
 * max_vectors and returns n. */
int or_last_krylov(const oracle_t* o, double* V, int max_vectors);

/* Time-dependent H, piecewise constant (replaced between steps): new hopping
 * scale J and site arrays eps, omega, g (NULL keeps one).  The move graph is
 * fixed: J and each g_s must stay zero exactly where they were (OR_INVALID). */
int or_set_coefficients(oracle_t* o, double J, const double* eps, const double* omega, const double* g);

/* hopping matrix J_ab the oracle built (N*N, row-major) */
void or_get_hopping(const oracle_t* o, double* out);

/* psi(0): n states given as site[n], occ[n*N] (A form), amps[2n] (re, im).
 * H_eff(0) is the ball of radius m_init (m_init < 0: closure) around them. */
int or_set_state(oracle_t* o, int n, const int* site, const int* occ, const double* amps);

/* A mid-trajectory state: n distinct rows (same form) with their amplitudes
 * become the current H_eff and vector exactly as a completed step leaves them,
 * so the next step truncates and regrows from them.  psi(0), the reference of
 * C(t), and the time are kept. */
int or_load_state(oracle_t* o, int n, const int* site, const int* occ, const double* amps);

/* One time step.  keep_override (length = rows before the step, or NULL)
 * replaces the threshold decision row by row. */
int or_step(oracle_t* o, double dt, double theta, const unsigned char* keep_override,
            int keep_len);

/* One time step with top-q_nom truncation (the q_nom rows of largest weight,
 * degenerate weights ordered by a seeded counter-based hash; see
 * paces_oracle.c).  The first step after set_state does not truncate. */
int or_step_nom(oracle_t* o, double dt, long long q_nom, unsigned long long seed);
/* The keep mask that step would use on the current rows (keep[nrows]). */
int or_nom_keep(const oracle_t* o, long long q_nom, unsigned long long seed, unsigned char* keep);
/* The tie-break hash u of a tuple (s, n_0..n_{N-1}) at step index t. */
unsigned long long or_tie_hash(unsigned long long seed, long long t, const int* tuple, int len);

int or_nrows(const oracle_t* o);
/* tuples[nrows*(N+1)] as (s, n_0..n_{N-1}); amps[2*nrows] */
void or_get_rows(const oracle_t* o, int* tuples, double* amps);
/* BFS level boundaries of the current H_eff: returns count, fills off[count] */
int or_level_offsets(const oracle_t* o, int* off, int max);
/* keep mask of the last truncation (over the rows before that step) */
int or_last_keep(const oracle_t* o, unsigned char* keep, int max);

/* P H P of the current H_eff.  Returns the number of off-diagonal entries;
 * if the pointers are non-NULL fills cnt[nrows], cols[], vals[], diag[nrows]
 * (entries of each row in move order). */
long or_build_hamiltonian(oracle_t* o, int* cnt, int* cols, double* vals, double* diag);

/* statistics of the last step (or of set_state), see OR_ST_* */
#define OR_ST_NORM 0        /* ||c||^2 after the step                     */
#define OR_ST_NORM_PHI0 1   /* ||c'||^2 entering the propagator            */
#define OR_ST_ENERGY 2      /* <c'|H_P|c'>                                */
#define OR_ST_C_RE 3        /* <psi0|psi(t)>                              */
#define OR_ST_C_IM 4
#define OR_ST_ROWS 5        /* q = dim H_eff                              */
#define OR_ST_KEPT 6        /* |M|                                        */
#define OR_ST_NNZ 7         /* off-diagonal entries + q diagonal entries   */
#define OR_ST_TERMS 8       /* Taylor terms used                          */
#define OR_ST_NORM_BEFORE 9 /* ||c||^2 before truncation                  */
#define OR_ST_TIME 10
#define OR_ST_SUBSTEPS 11   /* Taylor series the step was split into       */
#define OR_ST_HBOUND 12     /* bound rho on ||P H P|| used to split it      */
#define OR_NST 13
void or_stats(const oracle_t* o, double* st);
/* populations P_s[N] and mean phonon numbers nbar_j[N] of the current state */
void or_populations(const oracle_t* o, double* P, double* nbar);

/* adjoint: see paces_oracle.c (Sec. on gradients) */
int or_record(oracle_t* o, int on);
int or_backward(oracle_t* o, int nsteps_rec, const double* dL_dc_final /*2*nrows or NULL*/,
                const double* dL_dC /*2*(nsteps_rec) or NULL*/,
                const double* dL_dP /*N*(nsteps_rec) or NULL*/, double* grad /*3+N*/);

#ifdef __cplusplus
}
#endif
#endif
