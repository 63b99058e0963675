/*
 * paces_oracle.c -- plain FP64 CPU oracle of the co-evolving-subspace time step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  No code, table or
 * helper is shared with the CUDA library.
 *
 * What it computes (paces paper, arXiv 2603.07341):
 *   model      H = sum_s eps_s|s><s| + sum_{a!=b} J_ab|a><b|
 *                + sum_j omega_j n_j + sum_s g_s|s><s|(a_s^dag + a_s)      (Eq. holstein)
 *              with a hard phonon cap n_j <= K_j (App. parameters: d_pho - 1).
 *   neighbours N_M = {n : <n|H|m> != 0, m in M}; H_eff = ball of radius m in the
 *              graph H induces on basis states (Eqs. def_neighbor, def_neighbor_k, H_eff).
 *   one step   truncate by weight, regrow H_eff, rescue re-admitted amplitudes
 *              (Sec. "Truncation & post-adaptation detruncation"), build P H P
 *              (Sec. "Generating the effective Hamiltonian"), propagate with the
 *              Taylor series of exp(-i P H P dt) (App. C.1), record observables.
 *
 * Readings taken where the paper is silent:
 *   - truncation keeps a row iff re^2 + im^2 >= theta^2, evaluated in FP64 with
 *     no contraction (this file is compiled with -ffp-contract=off);
 *   - no truncation before the first propagation after set_state;
 *   - Taylor stops at the first n >= 2 with ||phi_n||^2 <= tol^2 ||r||^2;
 *   - row order: the kept set M in ascending basis order (n_{N-1} most
 *     significant, down to n_0, then s: the order of the paper's sorted key
 *     array), then every BFS level in first-occurrence order under the move
 *     order hops to t = 0..N-1 ascending, a_s^dag, a_s.
 *
 * Representation: a basis state is the int tuple (s, n_0, ..., n_{N-1}); rows
 * of H_eff are stored in order in a growable array with a linear-probing index.
 *
 * Propagators: the Taylor series of App. C.1 (default) or the Lanczos
 * decomposition of App. C.3 (or_set_propagator), with the same substep split.
 *
 * Planted mistakes: the pin tests compile this file a second time with one of
 * the macros OR_MUTANT_NO_RESCUE, OR_MUTANT_OPEN3D_AXES, OR_MUTANT_ENERGY_CONJ
 * or OR_MUTANT_LANCZOS_NO_BETA defined, each a plausible slip in one function,
 * and check that the pin of that function fails.  The default build defines
 * none of them.
 */
#include "paces_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ rowset */

typedef struct {
    int len;            /* ints per tuple = N + 1           */
    int nrows, cap;     /* rows stored, rows allocated      */
    int* t;             /* nrows * len                      */
    int* idx;           /* hash index: slot -> row, -1 empty */
    long nslots;        /* power of two                     */
} rowset;

static unsigned long long tuple_hash(const int* t, int len)
{
    /* FNV-1a over the integer values */
    unsigned long long h = 1469598103934665603ULL;
    for (int i = 0; i < len; ++i) {
        h ^= (unsigned long long)(unsigned int)t[i];
        h *= 1099511628211ULL;
    }
    return h ^ (h >> 29);
}

static int rs_init(rowset* r, int len)
{
    r->len = len;
    r->nrows = 0;
    r->cap = 64;
    r->t = (int*)malloc(sizeof(int) * (size_t)r->cap * (size_t)len);
    r->nslots = 128;
    r->idx = (int*)malloc(sizeof(int) * (size_t)r->nslots);
    if (!r->t || !r->idx) return OR_NOMEM;
    for (long i = 0; i < r->nslots; ++i) r->idx[i] = -1;
    return OR_OK;
}

static void rs_free(rowset* r)
{
    free(r->t);
    free(r->idx);
    r->t = NULL;
    r->idx = NULL;
    r->nrows = r->cap = 0;
}

static const int* rs_row(const rowset* r, int i) { return r->t + (size_t)i * (size_t)r->len; }

static int rs_find(const rowset* r, const int* tup)
{
    long mask = r->nslots - 1;
    long pos = (long)(tuple_hash(tup, r->len) & (unsigned long long)mask);
    for (;;) {
        int row = r->idx[pos];
        if (row < 0) return -1;
        if (memcmp(rs_row(r, row), tup, sizeof(int) * (size_t)r->len) == 0) return row;
        pos = (pos + 1) & mask;
    }
}

static void rs_place(rowset* r, int row)
{
    long mask = r->nslots - 1;
    long pos = (long)(tuple_hash(rs_row(r, row), r->len) & (unsigned long long)mask);
    while (r->idx[pos] >= 0) pos = (pos + 1) & mask;
    r->idx[pos] = row;
}

/* append a tuple known to be absent; returns its row or -1 on allocation failure */
static int rs_add(rowset* r, const int* tup)
{
    if (r->nrows == r->cap) {
        int ncap = r->cap * 2;
        int* nt = (int*)realloc(r->t, sizeof(int) * (size_t)ncap * (size_t)r->len);
        if (!nt) return -1;
        r->t = nt;
        r->cap = ncap;
    }
    memcpy(r->t + (size_t)r->nrows * (size_t)r->len, tup, sizeof(int) * (size_t)r->len);
    int row = r->nrows++;
    if (2L * r->nrows > r->nslots) {
        long ns = r->nslots * 2;
        int* ni = (int*)malloc(sizeof(int) * (size_t)ns);
        if (!ni) return -1;
        free(r->idx);
        r->idx = ni;
        r->nslots = ns;
        for (long i = 0; i < ns; ++i) r->idx[i] = -1;
        for (int i = 0; i < r->nrows; ++i) rs_place(r, i);
    } else {
        rs_place(r, row);
    }
    return row;
}

/* ------------------------------------------------------------------ oracle */

typedef struct {         /* one recorded step, for the adjoint */
    int nrows;
    int* tuples;         /* rows of H_eff of that step          */
    int* from;           /* rescue map: new row -> previous row or -1 */
    int nprev;
    cplx* cprime;        /* amplitudes entering the propagator  */
    int nterms;          /* terms over all substeps             */
    int nsub;            /* series the step was split into      */
    int* sub_terms;      /* terms of each series                */
    double dt;
} step_rec;

struct oracle {
    int N, len;
    double* Jm;          /* N*N hopping matrix J_ab              */
    double* Mm;          /* N*N hopping pattern dJ_ab/dJ          */
    double *eps, *omega, *g;
    int* cap;
    int m, m_init;
    double tol;
    int nmax, fixed_terms;
    double xmax;         /* substepping: series length bound rho dt / s <= xmax */
    int prop;            /* propagator: 0 Taylor series, 1 Lanczos (App. C.3)  */
    int kmax;            /* Lanczos: largest Krylov dimension                  */
    cplx* kry;           /* Lanczos basis v_1..v_n of the last series, q each  */
    int kry_n, kry_q;

    rowset rows;         /* current H_eff                         */
    cplx* c;             /* amplitudes on rows                    */
    int ccap;
    int fresh;           /* set_state done, first step not yet    */
    int tstep;           /* steps taken since set_state           */
    int* lvl;            /* BFS level offsets                     */
    int nlvl, lvlcap;
    unsigned char* keep; /* last truncation mask                  */
    int nkeep;

    /* P H P of the current rows */
    int hp_rows;
    int* hp_off;
    int* hp_col;
    double* hp_val;
    double* hp_dJ;       /* dH/dJ per entry                       */
    double* hp_dg;       /* dH/dg per entry                       */
    double* diag;
    long hp_nnz;

    rowset init;         /* psi(0) */
    cplx* c0;

    double st[OR_NST];
    double time;

    int recording;
    step_rec* rec;
    int nrec, reccap;
    int* last_from;      /* rescue map of the last step           */
};

static double hop_pattern(int lattice_kind, int coupling_kind, const int* dims, int N,
                          int a, int b)
{
    /* pattern M_ab such that J_ab = J * M_ab */
    if (a == b) return 0.0;
    if (lattice_kind == 0) {          /* ring: (j, j+1 mod N), pairs de-duplicated */
        if (N < 2) return 0.0;
        if ((a + 1) % N == b || (b + 1) % N == a) return 1.0;
        return 0.0;
    }
    int d0 = 1, d1 = 1;
    if (lattice_kind == 1) { d0 = N; d1 = 1; }
    if (lattice_kind == 2) { d0 = dims[0]; d1 = dims[1]; }
    if (lattice_kind == 3) { d0 = dims[0]; d1 = dims[1]; }
#ifdef OR_MUTANT_OPEN3D_AXES
    int t0 = d0; d0 = d1; d1 = t0;   /* planted: the two inner extents exchanged */
#endif
    int ax = a % d0, ay = (a / d0) % d1, az = a / (d0 * d1);
    int bx = b % d0, by = (b / d0) % d1, bz = b / (d0 * d1);
    double dx = ax - bx, dy = ay - by, dz = az - bz;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (coupling_kind == 0) return r2 == 1.0 ? 1.0 : 0.0;
    return 1.0 / (r2 * sqrt(r2));
}

oracle_t* or_create(int n_sites, int lattice_kind, const int* dims, int coupling_kind,
                    double J, const double* J_explicit, const double* eps,
                    const double* omega, const double* g, const int* cap,
                    int m, int m_init, double tol, int nmax, int fixed_terms)
{
    if (n_sites < 1 || lattice_kind < 0 || lattice_kind > 4 || coupling_kind < 0 ||
        coupling_kind > 1 || m < 0 || !cap)
        return NULL;
    if (lattice_kind == 2 && (!dims || dims[0] * dims[1] != n_sites)) return NULL;
    if (lattice_kind == 3 && (!dims || dims[0] * dims[1] * dims[2] != n_sites)) return NULL;
    if (lattice_kind == 4 && !J_explicit) return NULL;
    if (lattice_kind == 0 && coupling_kind != 0) return NULL;

    oracle_t* o = (oracle_t*)calloc(1, sizeof(oracle_t));
    if (!o) return NULL;
    int N = n_sites;
    o->N = N;
    o->len = N + 1;
    o->Jm = (double*)calloc((size_t)N * N, sizeof(double));
    o->Mm = (double*)calloc((size_t)N * N, sizeof(double));
    o->eps = (double*)calloc((size_t)N, sizeof(double));
    o->omega = (double*)calloc((size_t)N, sizeof(double));
    o->g = (double*)calloc((size_t)N, sizeof(double));
    o->cap = (int*)calloc((size_t)N, sizeof(int));
    for (int a = 0; a < N; ++a) {
        for (int b = 0; b < N; ++b) {
            double p;
            if (lattice_kind == 4) p = (a == b) ? 0.0 : J_explicit[a * N + b];
            else p = hop_pattern(lattice_kind, coupling_kind, dims, N, a, b);
            o->Mm[a * N + b] = p;
            o->Jm[a * N + b] = J * p;
        }
        o->eps[a] = eps ? eps[a] : 0.0;
        o->omega[a] = omega ? omega[a] : 0.0;
        o->g[a] = g ? g[a] : 0.0;
        o->cap[a] = cap[a];
        if (cap[a] < 0) { or_destroy(o); return NULL; }
    }
    o->m = m;
    o->m_init = m_init;
    o->tol = tol;
    o->nmax = nmax;
    o->fixed_terms = fixed_terms;
    o->xmax = 8.0;
    o->prop = 0;
    o->kmax = 30;
    rs_init(&o->rows, o->len);
    rs_init(&o->init, o->len);
    o->lvlcap = 64;
    o->lvl = (int*)malloc(sizeof(int) * (size_t)o->lvlcap);
    return o;
}

int or_set_xmax(oracle_t* o, double xmax)
{
    if (!o) return OR_INVALID;
    o->xmax = xmax;
    return OR_OK;
}

/* Piecewise-constant time dependence (Sec. 6's extension to time-dependent H:
 * the Hamiltonian is replaced between steps).  New values of J (the hopping
 * scale of the fixed pattern), eps, omega and g (NULL keeps an array); the
 * graph of moves may not change, so J and every g_s must stay zero exactly
 * where they were zero. */
int or_set_coefficients(oracle_t* o, double J, const double* eps, const double* omega, const double* g)
{
    if (!o || !isfinite(J)) return OR_INVALID;
    if (o->recording) return OR_INVALID;      /* the adjoint assumes one H for all steps */
    int N = o->N;
    int jz_old = 1;
    for (int i = 0; i < N * N; ++i)
        if (o->Jm[i] != 0.0) jz_old = 0;
    if ((J == 0.0) != jz_old) return OR_INVALID;
    for (int s = 0; s < N; ++s) {
        if (eps && !isfinite(eps[s])) return OR_INVALID;
        if (omega && !isfinite(omega[s])) return OR_INVALID;
        if (g && (!isfinite(g[s]) || ((g[s] == 0.0) != (o->g[s] == 0.0)))) return OR_INVALID;
    }
    for (int i = 0; i < N * N; ++i) o->Jm[i] = J * o->Mm[i];
    for (int s = 0; s < N; ++s) {
        if (eps) o->eps[s] = eps[s];
        if (omega) o->omega[s] = omega[s];
        if (g) o->g[s] = g[s];
    }
    return OR_OK;
}

int or_set_propagator(oracle_t* o, int kind, int kmax)
{
    if (!o || kind < 0 || kind > 1 || (kind == 1 && (kmax < 1 || kmax > OR_MAX_KRYLOV))) return OR_INVALID;
    if (kind == 1 && o->recording) return OR_INVALID;
    o->prop = kind;
    if (kind == 1) o->kmax = kmax;
    return OR_OK;
}

static void free_recs(oracle_t* o)
{
    for (int i = 0; i < o->nrec; ++i) {
        free(o->rec[i].sub_terms);
        free(o->rec[i].tuples);
        free(o->rec[i].from);
        free(o->rec[i].cprime);
    }
    free(o->rec);
    o->rec = NULL;
    o->nrec = o->reccap = 0;
}

void or_destroy(oracle_t* o)
{
    if (!o) return;
    free(o->Jm); free(o->Mm); free(o->eps); free(o->omega); free(o->g); free(o->cap);
    rs_free(&o->rows);
    rs_free(&o->init);
    free(o->c); free(o->c0); free(o->lvl); free(o->keep);
    free(o->hp_off); free(o->hp_col); free(o->hp_val); free(o->hp_dJ); free(o->hp_dg);
    free(o->diag);
    free(o->kry);
    free(o->last_from);
    free_recs(o);
    free(o);
}

void or_get_hopping(const oracle_t* o, double* out)
{
    memcpy(out, o->Jm, sizeof(double) * (size_t)o->N * (size_t)o->N);
}

/* Moves of basis state tup in canonical order.  Writes child tuples and the
 * matrix element <child|H|tup> (and its J and g derivatives); returns count. */
static int moves(const oracle_t* o, const int* tup, int* child, double* val, double* dJ,
                 double* dg)
{
    int N = o->N, len = o->len, s = tup[0], k = 0;
    for (int t = 0; t < N; ++t) {
        if (t == s || o->Jm[t * N + s] == 0.0) continue;
        memcpy(child + k * len, tup, sizeof(int) * (size_t)len);
        child[k * len] = t;
        val[k] = o->Jm[t * N + s];
        if (dJ) dJ[k] = o->Mm[t * N + s];
        if (dg) dg[k] = 0.0;
        ++k;
    }
    int ns = tup[1 + s];
    if (o->g[s] != 0.0 && ns < o->cap[s]) {             /* a_s^dag */
        memcpy(child + k * len, tup, sizeof(int) * (size_t)len);
        child[k * len + 1 + s] = ns + 1;
        val[k] = o->g[s] * sqrt((double)(ns + 1));
        if (dJ) dJ[k] = 0.0;
        if (dg) dg[k] = sqrt((double)(ns + 1));
        ++k;
    }
    if (o->g[s] != 0.0 && ns > 0) {                      /* a_s */
        memcpy(child + k * len, tup, sizeof(int) * (size_t)len);
        child[k * len + 1 + s] = ns - 1;
        val[k] = o->g[s] * sqrt((double)ns);
        if (dJ) dJ[k] = 0.0;
        if (dg) dg[k] = sqrt((double)ns);
        ++k;
    }
    return k;
}

static int max_moves(const oracle_t* o) { return o->N + 2; }

static double diag_of(const oracle_t* o, const int* tup)
{
    double d = o->eps[tup[0]];
    for (int j = 0; j < o->N; ++j) d = d + o->omega[j] * (double)tup[1 + j];
    return d;
}

static void lvl_push(oracle_t* o, int v)
{
    if (o->nlvl == o->lvlcap) {
        o->lvlcap *= 2;
        o->lvl = (int*)realloc(o->lvl, sizeof(int) * (size_t)o->lvlcap);
    }
    o->lvl[o->nlvl++] = v;
}

/* Grow rows by BFS levels: levels < 0 means until nothing new appears. */
static int expand(oracle_t* o, int levels)
{
    int len = o->len, D = max_moves(o);
    int* child = (int*)malloc(sizeof(int) * (size_t)D * (size_t)len);
    double* val = (double*)malloc(sizeof(double) * (size_t)D);
    int* parent = (int*)malloc(sizeof(int) * (size_t)len);
    if (!child || !val || !parent) return OR_NOMEM;
    o->nlvl = 0;
    lvl_push(o, 0);
    lvl_push(o, o->rows.nrows);
    int lo = 0, hi = o->rows.nrows;
    for (int l = 0; levels < 0 || l < levels; ++l) {
        for (int p = lo; p < hi; ++p) {
            memcpy(parent, rs_row(&o->rows, p), sizeof(int) * (size_t)len);
            int k = moves(o, parent, child, val, NULL, NULL);
            for (int i = 0; i < k; ++i)
                if (rs_find(&o->rows, child + i * len) < 0)
                    if (rs_add(&o->rows, child + i * len) < 0) return OR_NOMEM;
        }
        lo = hi;
        hi = o->rows.nrows;
        lvl_push(o, hi);
        if (lo == hi) break;
    }
    free(child); free(val); free(parent);
    return OR_OK;
}

static int ensure_c(oracle_t* o, int n)
{
    if (n <= o->ccap) return OR_OK;
    int nc = o->ccap ? o->ccap : 64;
    while (nc < n) nc *= 2;
    cplx* c = (cplx*)realloc(o->c, sizeof(cplx) * (size_t)nc);
    if (!c) return OR_NOMEM;
    o->c = c;
    o->ccap = nc;
    return OR_OK;
}

static void observe(oracle_t* o);

int or_set_state(oracle_t* o, int n, const int* site, const int* occ, const double* amps)
{
    if (!o || n <= 0 || !site || !occ || !amps) return OR_INVALID;
    int N = o->N, len = o->len;
    rs_free(&o->rows);
    rs_free(&o->init);
    rs_init(&o->rows, len);
    rs_init(&o->init, len);
    free(o->c0);
    o->c0 = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    int* tup = (int*)malloc(sizeof(int) * (size_t)len);
    if (ensure_c(o, n)) return OR_NOMEM;
    for (int i = 0; i < n; ++i) {
        if (site[i] < 0 || site[i] >= N) { free(tup); return OR_INVALID; }
        tup[0] = site[i];
        for (int j = 0; j < N; ++j) {
            int v = occ[(size_t)i * N + j];
            if (v < 0 || v > o->cap[j]) { free(tup); return OR_INVALID; }
            tup[1 + j] = v;
        }
        if (rs_find(&o->rows, tup) >= 0) { free(tup); return OR_INVALID; }
        rs_add(&o->rows, tup);
        rs_add(&o->init, tup);
        o->c[i] = amps[2 * i] + I * amps[2 * i + 1];
        o->c0[i] = o->c[i];
    }
    free(tup);
    int rc = expand(o, o->m_init);
    if (rc) return rc;
    if (ensure_c(o, o->rows.nrows)) return OR_NOMEM;
    for (int i = n; i < o->rows.nrows; ++i) o->c[i] = 0.0;
    o->fresh = 1;
    o->tstep = 0;
    o->time = 0.0;
    free_recs(o);
    memset(o->st, 0, sizeof(o->st));
    observe(o);
    o->st[OR_ST_ROWS] = o->rows.nrows;
    o->st[OR_ST_KEPT] = n;
    o->st[OR_ST_NORM_PHI0] = o->st[OR_ST_NORM];
    o->st[OR_ST_NORM_BEFORE] = o->st[OR_ST_NORM];
    return OR_OK;
}

int or_load_state(oracle_t* o, int n, const int* site, const int* occ, const double* amps)
{
    if (!o || n <= 0 || !site || !occ || !amps) return OR_INVALID;
    int N = o->N, len = o->len;
    rs_free(&o->rows);
    rs_init(&o->rows, len);
    int* tup = (int*)malloc(sizeof(int) * (size_t)len);
    if (!tup || ensure_c(o, n)) { free(tup); return OR_NOMEM; }
    for (int i = 0; i < n; ++i) {
        if (site[i] < 0 || site[i] >= N) { free(tup); return OR_INVALID; }
        tup[0] = site[i];
        for (int j = 0; j < N; ++j) {
            int v = occ[(size_t)i * N + j];
            if (v < 0 || v > o->cap[j]) { free(tup); return OR_INVALID; }
            tup[1 + j] = v;
        }
        if (rs_find(&o->rows, tup) >= 0) { free(tup); return OR_INVALID; }
        if (rs_add(&o->rows, tup) < 0) { free(tup); return OR_NOMEM; }
        o->c[i] = amps[2 * i] + I * amps[2 * i + 1];
    }
    free(tup);
    o->fresh = 0;
    o->nlvl = 0;
    lvl_push(o, 0);
    lvl_push(o, n);
    free(o->keep);
    o->keep = NULL;
    o->nkeep = 0;
    free(o->last_from);
    o->last_from = NULL;
    free_recs(o);
    observe(o);
    o->st[OR_ST_ROWS] = n;
    o->st[OR_ST_KEPT] = n;
    o->st[OR_ST_NORM_PHI0] = o->st[OR_ST_NORM];
    o->st[OR_ST_NORM_BEFORE] = o->st[OR_ST_NORM];
    return OR_OK;
}

long or_build_hamiltonian(oracle_t* o, int* cnt, int* cols, double* vals, double* diag)
{
    int q = o->rows.nrows, len = o->len, D = max_moves(o);
    free(o->hp_off); free(o->hp_col); free(o->hp_val); free(o->hp_dJ); free(o->hp_dg);
    free(o->diag);
    o->hp_off = (int*)malloc(sizeof(int) * ((size_t)q + 1));
    o->hp_col = (int*)malloc(sizeof(int) * ((size_t)q * D + 1));
    o->hp_val = (double*)malloc(sizeof(double) * ((size_t)q * D + 1));
    o->hp_dJ = (double*)malloc(sizeof(double) * ((size_t)q * D + 1));
    o->hp_dg = (double*)malloc(sizeof(double) * ((size_t)q * D + 1));
    o->diag = (double*)malloc(sizeof(double) * ((size_t)q + 1));
    int* child = (int*)malloc(sizeof(int) * (size_t)D * (size_t)len);
    double* val = (double*)malloc(sizeof(double) * (size_t)D);
    double* dJ = (double*)malloc(sizeof(double) * (size_t)D);
    double* dg = (double*)malloc(sizeof(double) * (size_t)D);
    long nnz = 0;
    for (int i = 0; i < q; ++i) {
        const int* tup = rs_row(&o->rows, i);
        o->hp_off[i] = (int)nnz;
        o->diag[i] = diag_of(o, tup);
        int k = moves(o, tup, child, val, dJ, dg);
        for (int e = 0; e < k; ++e) {
            int j = rs_find(&o->rows, child + e * len);
            if (j < 0) continue;                  /* image outside H_eff */
            o->hp_col[nnz] = j;
            o->hp_val[nnz] = val[e];
            o->hp_dJ[nnz] = dJ[e];
            o->hp_dg[nnz] = dg[e];
            ++nnz;
        }
    }
    o->hp_off[q] = (int)nnz;
    o->hp_rows = q;
    o->hp_nnz = nnz;
    free(child); free(val); free(dJ); free(dg);
    if (cnt) for (int i = 0; i < q; ++i) cnt[i] = o->hp_off[i + 1] - o->hp_off[i];
    if (cols) memcpy(cols, o->hp_col, sizeof(int) * (size_t)nnz);
    if (vals) memcpy(vals, o->hp_val, sizeof(double) * (size_t)nnz);
    if (diag) memcpy(diag, o->diag, sizeof(double) * (size_t)q);
    return nnz;
}

/* y = P H P x */
static void apply_h(const oracle_t* o, const cplx* x, cplx* y)
{
    for (int i = 0; i < o->hp_rows; ++i) {
        cplx acc = o->diag[i] * x[i];
        for (int e = o->hp_off[i]; e < o->hp_off[i + 1]; ++e) acc += o->hp_val[e] * x[o->hp_col[e]];
        y[i] = acc;
    }
}

static double norm2(const cplx* v, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return s;
}

/* Bound rho on ||P H P||_2: the largest absolute row sum of H over the rows of
 * H_eff (a row sum of H bounds that of P H P, and for a Hermitian matrix the
 * largest row sum bounds the spectral norm).  Each term is rounded up to a
 * multiple of 2^-20 and the terms are added as integers, so the value does not
 * depend on the order of the additions. */
static unsigned long long up20(double x) { return (unsigned long long)ceil(fabs(x) * 1048576.0); }

static unsigned long long row_bound(const oracle_t* o, const int* t)
{
    int N = o->N, s = t[0], ns = t[1 + s];
    unsigned long long b = up20(o->eps[s]);
    for (int j = 0; j < N; ++j) b += up20(o->omega[j]) * (unsigned long long)t[1 + j];
    for (int u = 0; u < N; ++u)
        if (u != s) b += up20(o->Jm[u * N + s]);
    if (o->g[s] != 0.0) {
        if (ns < o->cap[s]) b += up20(o->g[s] * sqrt((double)(ns + 1)));
        if (ns > 0) b += up20(o->g[s] * sqrt((double)ns));
    }
    return b;
}

#define OR_MAX_SUB 1024

/* Number of series a step of length dt is split into: s = ceil(rho dt / xmax)
 * (1 when xmax <= 0).  0 when more than OR_MAX_SUB would be needed. */
static int substeps(const oracle_t* o, double dt, double* rho_out)
{
    unsigned long long rb = 0;
    for (int i = 0; i < o->rows.nrows; ++i) {
        unsigned long long b = row_bound(o, rs_row(&o->rows, i));
        if (b > rb) rb = b;
    }
    double rho = (double)rb / 1048576.0;
    *rho_out = rho;
    if (o->xmax <= 0.0) return 1;
    double ns = ceil(rho * dt / o->xmax);
    if (ns > (double)OR_MAX_SUB) return 0;
    return ns < 1.0 ? 1 : (int)ns;
}

/* c <- exp(-i dt H_P) c as nsub successive Taylor series of length h = dt/nsub,
 * each r = sum_n (-i h H)^n / n! v via phi_n = (-i h / n) H phi_{n-1}
 * (App. C.1), stopping at the first n >= 2 with ||phi_n||^2 <= tol^2 ||r||^2.
 * sub_terms[j] receives the terms of series j; energy = <c|H_P|c> of the input. */
static int taylor(oracle_t* o, double dt, int nsub, cplx* c, int* sub_terms, int* nterms_out, double* energy)
{
    int q = o->hp_rows;
    cplx* phi = (cplx*)malloc(sizeof(cplx) * ((size_t)q + 1));
    cplx* y = (cplx*)malloc(sizeof(cplx) * ((size_t)q + 1));
    cplx* r = (cplx*)malloc(sizeof(cplx) * ((size_t)q + 1));
    if (!phi || !y || !r) return OR_NOMEM;
    double h = dt / (double)nsub;
    int converged = 1, total = 0;
    int nlimit = o->fixed_terms > 0 ? o->fixed_terms : o->nmax;
    *energy = 0.0;
    for (int j = 0; j < nsub && converged; ++j) {
        memcpy(phi, c, sizeof(cplx) * (size_t)q);
        memcpy(r, c, sizeof(cplx) * (size_t)q);
        int done = 0, n = 0;
        for (n = 1; n <= nlimit; ++n) {
            apply_h(o, phi, y);
            if (j == 0 && n == 1) {
                double e = 0.0;
#ifdef OR_MUTANT_ENERGY_CONJ
                for (int i = 0; i < q; ++i) e += creal(c[i] * y[i]);        /* planted: conj dropped */
#else
                for (int i = 0; i < q; ++i) e += creal(conj(c[i]) * y[i]);
#endif
                *energy = e;
            }
            cplx f = -I * h / (double)n;
            for (int i = 0; i < q; ++i) {
                phi[i] = f * y[i];
                r[i] += phi[i];
            }
            if (o->fixed_terms > 0) continue;
            double a = norm2(phi, q), b = norm2(r, q);
            if (n >= 2 && a <= o->tol * o->tol * b) { done = 1; break; }
        }
        if (o->fixed_terms > 0) { done = 1; n = o->fixed_terms; }
        if (!done) { converged = 0; n = nlimit; }
        if (sub_terms) sub_terms[j] = n;
        total += n;
        memcpy(c, r, sizeof(cplx) * (size_t)q);
    }
    free(phi); free(y); free(r);
    *nterms_out = total;
    return converged ? OR_OK : OR_NOCONVERGE;
}

/* ------------------------------------------------------------------ Lanczos */

/* Eigen-decomposition of the real symmetric n x n matrix A (row-major, n <=
 * OR_MAX_KRYLOV) by cyclic Jacobi rotations: on return the diagonal of A holds
 * the eigenvalues and column k of Q (row-major) the eigenvector of A[k][k]. */
static void jacobi_eigen(double* A, double* Q, int n)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Q[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-34 * tot || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                /* rotation angle that zeroes A[p][q] */
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {          /* A <- A G (columns p, q) */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          /* A <- G^T A (rows p, q) */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {          /* Q <- Q G */
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - sn * qkq;
                    Q[k * n + q] = sn * qkp + c * qkq;
                }
            }
    }
}

/* y = exp(-i h T) e_1 for the n x n symmetric tridiagonal T with diagonal
 * alpha[0..n-1] and off-diagonal beta[0..n-2], through T = Q diag(lambda) Q^T. */
static void tridiag_exp_e1(const double* alpha, const double* beta, int n, double h, cplx* y)
{
    double A[OR_MAX_KRYLOV * OR_MAX_KRYLOV], Q[OR_MAX_KRYLOV * OR_MAX_KRYLOV];
    for (int i = 0; i < n * n; ++i) A[i] = 0.0;
    for (int i = 0; i < n; ++i) {
        A[i * n + i] = alpha[i];
        if (i + 1 < n) A[i * n + i + 1] = A[(i + 1) * n + i] = beta[i];
    }
    jacobi_eigen(A, Q, n);
    for (int i = 0; i < n; ++i) {
        cplx acc = 0.0;
        for (int k = 0; k < n; ++k) acc += Q[i * n + k] * cexp(-I * h * A[k * n + k]) * Q[0 * n + k];
        y[i] = acc;
    }
}

/* c <- exp(-i dt H_P) c by the Lanczos decomposition of App. C.3,
 * exp(-i h H) v ~ V_n exp(-i h T_n) V_n^dag v = beta_0 V_n exp(-i h T_n) e_1,
 * as nsub successive decompositions of length h = dt / nsub.  The three-term
 * recurrence: v_1 = v / beta_0 (beta_0 = ||v||); for j = 1, 2, ..:
 * w = H v_j, alpha_j = <v_j|w>, w -= alpha_j v_j + beta_{j-1} v_{j-1},
 * beta_j = ||w||, v_{j+1} = w / beta_j.  It stops at the first j whose error
 * estimate h beta_j |(exp(-i h T_j) e_1)_j| (the norm of the residual of the
 * Krylov solution, relative to ||v||, times h) is <= tol, and fails past
 * kmax vectors.  sub_terms[j]: the dimension n of series j (= applications of
 * H); energy = <c|H_P|c> of the input = beta_0^2 alpha_1.  The basis of the
 * last series stays in o->kry. */
static int lanczos(oracle_t* o, double dt, int nsub, cplx* c, int* sub_terms, int* nterms_out, double* energy)
{
    int q = o->hp_rows, K = o->kmax;
    free(o->kry);
    o->kry = (cplx*)malloc(sizeof(cplx) * ((size_t)q * (size_t)(K + 1) + 1));
    cplx* w = (cplx*)malloc(sizeof(cplx) * ((size_t)q + 1));
    if (!o->kry || !w) { free(w); return OR_NOMEM; }
    double h = dt / (double)nsub;
    double alpha[OR_MAX_KRYLOV], beta[OR_MAX_KRYLOV + 1];
    cplx y[OR_MAX_KRYLOV];
    int converged = 1, total = 0;
    *energy = 0.0;
    o->kry_n = 0;
    o->kry_q = q;
    for (int js = 0; js < nsub && converged; ++js) {
        double b0 = sqrt(norm2(c, q));
        if (b0 == 0.0) {              /* zero vector: exp(..) 0 = 0 */
            if (sub_terms) sub_terms[js] = 0;
            o->kry_n = 0;
            continue;
        }
        cplx* V = o->kry;
        for (int i = 0; i < q; ++i) V[i] = c[i] / b0;
        int n = 0, done = 0;
        for (int j = 1; j <= K; ++j) {
            cplx* vj = V + (size_t)(j - 1) * q;
            apply_h(o, vj, w);
            double a = 0.0;
            for (int i = 0; i < q; ++i) a += creal(conj(vj[i]) * w[i]);
            alpha[j - 1] = a;
            if (js == 0 && j == 1) *energy = b0 * b0 * a;
            for (int i = 0; i < q; ++i) {
                w[i] -= a * vj[i];
#ifndef OR_MUTANT_LANCZOS_NO_BETA
                if (j > 1) w[i] -= beta[j - 1] * V[(size_t)(j - 2) * q + i];
#endif
            }
            double bj = sqrt(norm2(w, q));
            beta[j] = bj;
            /* T_j: diagonal alpha_1..alpha_j, off-diagonal beta_1..beta_{j-1} */
            tridiag_exp_e1(alpha, beta + 1, j, h, y);
            n = j;
            if (h * bj * cabs(y[j - 1]) <= o->tol) { done = 1; break; }
            if (j < K)
                for (int i = 0; i < q; ++i) V[(size_t)j * q + i] = w[i] / bj;
        }
        if (!done) { converged = 0; n = K; }
        if (sub_terms) sub_terms[js] = n;
        total += n;
        o->kry_n = n;
        if (done)
            for (int i = 0; i < q; ++i) {
                cplx acc = 0.0;
                for (int k = 0; k < n; ++k) acc += y[k] * V[(size_t)k * q + i];
                c[i] = b0 * acc;
            }
    }
    free(w);
    *nterms_out = total;
    return converged ? OR_OK : OR_NOCONVERGE;
}

int or_last_krylov(const oracle_t* o, double* V, int max_vectors)
{
    if (!o || !o->kry) return 0;
    int n = o->kry_n < max_vectors ? o->kry_n : max_vectors;
    if (V)
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < o->kry_q; ++i) {
                V[2 * ((size_t)k * o->kry_q + i)] = creal(o->kry[(size_t)k * o->kry_q + i]);
                V[2 * ((size_t)k * o->kry_q + i) + 1] = cimag(o->kry[(size_t)k * o->kry_q + i]);
            }
    return o->kry_n;
}

static void observe(oracle_t* o)
{
    int q = o->rows.nrows;
    o->st[OR_ST_NORM] = norm2(o->c, q);
    cplx ov = 0.0;
    for (int k = 0; k < o->init.nrows; ++k) {
        int j = rs_find(&o->rows, rs_row(&o->init, k));
        if (j >= 0) ov += conj(o->c0[k]) * o->c[j];
    }
    o->st[OR_ST_C_RE] = creal(ov);
    o->st[OR_ST_C_IM] = cimag(ov);
    o->st[OR_ST_TIME] = o->time;
}

void or_populations(const oracle_t* o, double* P, double* nbar)
{
    int N = o->N;
    for (int j = 0; j < N; ++j) P[j] = nbar[j] = 0.0;
    for (int i = 0; i < o->rows.nrows; ++i) {
        const int* t = rs_row(&o->rows, i);
        double w = creal(o->c[i]) * creal(o->c[i]) + cimag(o->c[i]) * cimag(o->c[i]);
        P[t[0]] += w;
        for (int j = 0; j < N; ++j) nbar[j] += w * (double)t[1 + j];
    }
}

/* Sort row indices by basis state: n_{N-1} first, down to n_0, then s. */
static const rowset* g_sort_rows;
static int basis_cmp(const void* a, const void* b)
{
    const int* x = rs_row(g_sort_rows, *(const int*)a);
    const int* y = rs_row(g_sort_rows, *(const int*)b);
    int len = g_sort_rows->len;
    for (int j = len - 1; j >= 1; --j)
        if (x[j] != y[j]) return x[j] < y[j] ? -1 : 1;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return 0;
}

static void sort_rows_by_basis(const rowset* rows, int* idx, int n)
{
    g_sort_rows = rows;
    qsort(idx, (size_t)n, sizeof(int), basis_cmp);     /* states are distinct: no ties */
    g_sort_rows = NULL;
}

int or_step(oracle_t* o, double dt, double theta, const unsigned char* keep_override,
            int keep_len)
{
    if (!o || (o->rows.nrows == 0 && !o->fresh)) return OR_STATE;
    if (o->prop == 1 && o->recording) return OR_INVALID;
    int len = o->len;
    int q_old = o->rows.nrows;
    double norm_before = norm2(o->c, q_old);
    int kept = q_old;
    free(o->last_from);
    o->last_from = NULL;
    if (!o->fresh) {
        if (keep_override && keep_len != q_old) return OR_INVALID;
        /* 1. truncation Q: keep rows whose weight reaches theta^2 */
        free(o->keep);
        o->keep = (unsigned char*)malloc((size_t)q_old + 1);
        o->nkeep = q_old;
        double th2 = theta * theta;
        for (int i = 0; i < q_old; ++i) {
            double re = creal(o->c[i]), im = cimag(o->c[i]);
            double w = re * re + im * im;
            o->keep[i] = keep_override ? (keep_override[i] != 0) : (w >= th2);
        }
        /* 2. M in ascending basis order -- the tuple compared from n_{N-1}
         *    down to n_0, then s -- the order of the paper's sorted key array;
         *    then regrow H_eff by m BFS levels */
        rowset old = o->rows;
        cplx* cold = o->c;
        o->c = NULL;
        o->ccap = 0;
        rs_init(&o->rows, len);
        kept = 0;
        int* mi = (int*)malloc(sizeof(int) * ((size_t)q_old + 1));
        if (!mi) return OR_NOMEM;
        for (int i = 0; i < q_old; ++i)
            if (o->keep[i]) mi[kept++] = i;
        sort_rows_by_basis(&old, mi, kept);
        for (int i = 0; i < kept; ++i) rs_add(&o->rows, rs_row(&old, mi[i]));
        free(mi);
        int rc = expand(o, o->m);
        if (rc) return rc;
        /* 3. rescue: amplitudes of re-admitted states come back (detruncation) */
        int q = o->rows.nrows;
        if (ensure_c(o, q > 0 ? q : 1)) return OR_NOMEM;
        o->last_from = (int*)malloc(sizeof(int) * ((size_t)q + 1));
        for (int i = 0; i < q; ++i) {
            int j = rs_find(&old, rs_row(&o->rows, i));
            o->last_from[i] = j;
#ifdef OR_MUTANT_NO_RESCUE
            if (i >= kept) j = -1;          /* planted: re-admitted rows restart at 0 */
#endif
            o->c[i] = (j >= 0) ? cold[j] : 0.0;
        }
        rs_free(&old);
        free(cold);
    }
    /* 4. P H P, 5. propagation */
    or_build_hamiltonian(o, NULL, NULL, NULL, NULL);
    int q = o->rows.nrows;
    if (o->recording) {
        if (o->nrec == o->reccap) {
            o->reccap = o->reccap ? 2 * o->reccap : 16;
            o->rec = (step_rec*)realloc(o->rec, sizeof(step_rec) * (size_t)o->reccap);
        }
        step_rec* R = &o->rec[o->nrec++];
        memset(R, 0, sizeof(*R));
        R->nrows = q;
        R->tuples = (int*)malloc(sizeof(int) * (size_t)q * len + 1);
        memcpy(R->tuples, o->rows.t, sizeof(int) * (size_t)q * len);
        R->from = (int*)malloc(sizeof(int) * ((size_t)q + 1));
        for (int i = 0; i < q; ++i) R->from[i] = o->last_from ? o->last_from[i] : i;
        R->nprev = q_old;
        R->cprime = (cplx*)malloc(sizeof(cplx) * ((size_t)q + 1));
        memcpy(R->cprime, o->c, sizeof(cplx) * (size_t)q);
    }
    double n0 = norm2(o->c, q);
    int nterms = 0;
    double energy = 0.0, rho = 0.0;
    int nsub = substeps(o, dt, &rho);
    int* sub_terms = (int*)calloc((size_t)(nsub > 0 ? nsub : 1), sizeof(int));
    if (!sub_terms) return OR_NOMEM;
    int rc = nsub <= 0 ? OR_NOCONVERGE
           : o->prop == 1 ? lanczos(o, dt, nsub, o->c, sub_terms, &nterms, &energy)
                          : taylor(o, dt, nsub, o->c, sub_terms, &nterms, &energy);
    if (o->recording) {
        o->rec[o->nrec - 1].nterms = nterms;
        o->rec[o->nrec - 1].nsub = nsub;
        o->rec[o->nrec - 1].sub_terms = sub_terms;
        o->rec[o->nrec - 1].dt = dt;
    } else {
        free(sub_terms);
    }
    o->st[OR_ST_SUBSTEPS] = nsub;
    o->st[OR_ST_HBOUND] = rho;
    o->time += dt;
    o->fresh = 0;
    o->tstep += 1;
    observe(o);
    o->st[OR_ST_NORM_PHI0] = n0;
    o->st[OR_ST_ENERGY] = energy;
    o->st[OR_ST_ROWS] = q;
    o->st[OR_ST_KEPT] = kept;
    o->st[OR_ST_NNZ] = (double)(o->hp_nnz + q);
    o->st[OR_ST_TERMS] = nterms;
    o->st[OR_ST_NORM_BEFORE] = norm_before;
    return rc;
}

int or_nrows(const oracle_t* o) { return o->rows.nrows; }

void or_get_rows(const oracle_t* o, int* tuples, double* amps)
{
    int q = o->rows.nrows;
    if (tuples) memcpy(tuples, o->rows.t, sizeof(int) * (size_t)q * (size_t)o->len);
    if (amps)
        for (int i = 0; i < q; ++i) {
            amps[2 * i] = creal(o->c[i]);
            amps[2 * i + 1] = cimag(o->c[i]);
        }
}

int or_level_offsets(const oracle_t* o, int* off, int max)
{
    for (int i = 0; i < o->nlvl && i < max; ++i) off[i] = o->lvl[i];
    return o->nlvl;
}

int or_last_keep(const oracle_t* o, unsigned char* keep, int max)
{
    for (int i = 0; i < o->nkeep && i < max; ++i) keep[i] = o->keep[i];
    return o->nkeep;
}

void or_stats(const oracle_t* o, double* st) { memcpy(st, o->st, sizeof(o->st)); }

/* ------------------------------------------------------------------ top-q_nom
 *
 * Truncation to the q_nom basis states of largest weight w = re^2 + im^2 (the
 * paper's scheme: Sec. "Truncation & post-adaptation detruncation"; App. "How
 * to weight states for truncation").  The appendix warns that degenerate
 * weights cut in a fixed order bias the result and recommends randomising the
 * order of degenerate states at the cutoff.  Reading taken here: among equal
 * weights, states are ordered by a key
 *     tk = (u with its low 32 bits cleared) | (0xFFFFFFFF - row),
 * u = a counter-based hash of (seed, t, s, n_0, .., n_{N-1}):
 *     z = seed + G t,  z = mix(z xor v) for v = s, n_0, .., n_{N-1},  u = z,
 * with G = 0x9E3779B97F4A7C15 and mix the output function of SplitMix64
 * (Steele, Lea & Flood 2014), and t = 1 + the number of steps since
 * set_state.  Larger (w, tk) is kept first; tk is unique (it holds the row),
 * so exactly q_nom rows are kept whenever q > q_nom. */
static unsigned long long mix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

unsigned long long or_tie_hash(unsigned long long seed, long long t, const int* tuple, int len)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)t;
    for (int i = 0; i < len; ++i) z = mix64(z ^ (unsigned long long)(unsigned)tuple[i]);
    return z;
}

typedef struct {
    double w;
    unsigned long long tk;
    int row;
} nom_item;

static int nom_cmp(const void* a, const void* b)
{
    const nom_item* x = (const nom_item*)a;
    const nom_item* y = (const nom_item*)b;
    if (x->w != y->w) return x->w > y->w ? -1 : 1;
    if (x->tk != y->tk) return x->tk > y->tk ? -1 : 1;
    return 0;
}

int or_nom_keep(const oracle_t* o, long long q_nom, unsigned long long seed, unsigned char* keep)
{
    int q = o->rows.nrows;
    if (q_nom < 0) return OR_INVALID;
    if ((long long)q <= q_nom) {
        for (int i = 0; i < q; ++i) keep[i] = 1;
        return OR_OK;
    }
    nom_item* it = (nom_item*)malloc(sizeof(nom_item) * ((size_t)q + 1));
    if (!it) return OR_NOMEM;
    long long t = (long long)o->tstep + 1;
    for (int i = 0; i < q; ++i) {
        double re = creal(o->c[i]), im = cimag(o->c[i]);
        unsigned long long u = or_tie_hash(seed, t, rs_row(&o->rows, i), o->len);
        it[i].w = re * re + im * im;
        it[i].tk = (u & 0xFFFFFFFF00000000ULL) | (0xFFFFFFFFULL - (unsigned long long)(unsigned)i);
        it[i].row = i;
    }
    qsort(it, (size_t)q, sizeof(nom_item), nom_cmp);
    for (int i = 0; i < q; ++i) keep[i] = 0;
    for (long long i = 0; i < q_nom; ++i) keep[it[i].row] = 1;
    free(it);
    return OR_OK;
}

int or_step_nom(oracle_t* o, double dt, long long q_nom, unsigned long long seed)
{
    if (!o || (o->rows.nrows == 0 && !o->fresh)) return OR_STATE;
    if (q_nom < 0) return OR_INVALID;
    if (o->fresh) return or_step(o, dt, 0.0, NULL, 0);
    int q = o->rows.nrows;
    unsigned char* keep = (unsigned char*)malloc((size_t)q + 1);
    if (!keep) return OR_NOMEM;
    int rc = or_nom_keep(o, q_nom, seed, keep);
    if (rc == OR_OK) rc = or_step(o, dt, 0.0, keep, q);
    free(keep);
    return rc;
}

/* ------------------------------------------------------------------ adjoint
 *
 * Gradient of a real loss L of the recorded trajectory with respect to
 * theta = (J, g, omega, eps_0..eps_{N-1}), holding the recorded subspace
 * sequence and term counts fixed.  Cotangents use dL = Re(mu^dag dc).
 * For one step with phi_n = B_n phi_{n-1}, B_n = (-i dt/n) H, c = sum_n phi_n:
 *   mu_N = gbar, mu_{n-1} = gbar + B_n^dag mu_n,
 *   dL/dtheta_p += sum_n Re(mu_n^dag (-i dt/n) (dH/dtheta_p) phi_{n-1}),
 * and the cotangent of the previous step's amplitudes is mu_0 scattered back
 * through the rescue map.  H is linear in every parameter, so dH/dtheta_p has
 * the sparsity of H with the derivative coefficients.
 */
int or_record(oracle_t* o, int on)
{
    free_recs(o);
    o->recording = on;
    return OR_OK;
}

/* rebuild rows/hamiltonian of a recorded step into the oracle (scratch use) */
static int load_rec_rows(oracle_t* o, const step_rec* R)
{
    rs_free(&o->rows);
    rs_init(&o->rows, o->len);
    for (int i = 0; i < R->nrows; ++i)
        if (rs_add(&o->rows, R->tuples + (size_t)i * o->len) < 0) return OR_NOMEM;
    or_build_hamiltonian(o, NULL, NULL, NULL, NULL);
    return OR_OK;
}

/* y = (dH/dtheta_p) x for p = 0 (J), 1 (g), 2 (omega), 3+s (eps_s) */
static void apply_dh(const oracle_t* o, int p, const cplx* x, cplx* y)
{
    for (int i = 0; i < o->hp_rows; ++i) {
        const int* t = rs_row(&o->rows, i);
        cplx acc = 0.0;
        if (p == 0 || p == 1) {
            const double* d = (p == 0) ? o->hp_dJ : o->hp_dg;
            for (int e = o->hp_off[i]; e < o->hp_off[i + 1]; ++e) acc += d[e] * x[o->hp_col[e]];
        } else if (p == 2) {
            double nsum = 0.0;
            for (int j = 0; j < o->N; ++j) nsum += (double)t[1 + j];
            acc = nsum * x[i];
        } else {
            acc = (t[0] == p - 3) ? x[i] : 0.0;
        }
        y[i] = acc;
    }
}

int or_backward(oracle_t* o, int nsteps_rec, const double* dL_dc_final, const double* dL_dC,
                const double* dL_dP, double* grad)
{
    if (!o || nsteps_rec != o->nrec || nsteps_rec <= 0) return OR_INVALID;
    int N = o->N, len = o->len, P = 3 + N;
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    /* park the live state; the recorded steps are reloaded one by one */
    rowset live = o->rows;
    cplx* live_c = o->c;
    int live_ccap = o->ccap;
    o->c = NULL;
    o->ccap = 0;
    rs_init(&o->rows, len);

    const step_rec* last = &o->rec[nsteps_rec - 1];
    cplx* gbar = (cplx*)calloc((size_t)last->nrows + 1, sizeof(cplx));
    if (dL_dc_final)
        for (int i = 0; i < last->nrows; ++i)
            gbar[i] = dL_dc_final[2 * i] + I * dL_dc_final[2 * i + 1];

    int rc = OR_OK;
    for (int k = nsteps_rec - 1; k >= 0 && rc == OR_OK; --k) {
        const step_rec* R = &o->rec[k];
        int q = R->nrows;
        rc = load_rec_rows(o, R);
        if (rc) break;
        /* forward terms of this step, recomputed: series j of the step keeps
         * phi^(j)_0 .. phi^(j)_{n_j} at phis + (base_j + n) qs, phi^(j)_0 being
         * the input of series j (c' for j = 0, else the output of series j-1) */
        int ns = R->nsub;
        double h = R->dt / (double)ns;
        size_t qs = (size_t)q + 1;
        int* base = (int*)malloc(sizeof(int) * ((size_t)ns + 1));
        if (!base) { rc = OR_NOMEM; break; }
        base[0] = 0;
        for (int j = 0; j < ns; ++j) base[j + 1] = base[j] + R->sub_terms[j] + 1;
        cplx* phis = (cplx*)malloc(sizeof(cplx) * (size_t)base[ns] * qs);
        cplx* y = (cplx*)malloc(sizeof(cplx) * qs);
        cplx* mu = (cplx*)malloc(sizeof(cplx) * qs);
        if (!phis || !y || !mu) { rc = OR_NOMEM; break; }
        memcpy(phis, R->cprime, sizeof(cplx) * (size_t)q);
        for (int j = 0; j < ns; ++j) {
            cplx* ph = phis + (size_t)base[j] * qs;
            if (j > 0) {           /* input of series j = sum of the terms of series j-1 */
                const cplx* prv = phis + (size_t)base[j - 1] * qs;
                for (int i = 0; i < q; ++i) {
                    cplx v = 0.0;
                    for (int n = 0; n <= R->sub_terms[j - 1]; ++n) v += prv[(size_t)n * qs + i];
                    ph[i] = v;
                }
            }
            for (int n = 1; n <= R->sub_terms[j]; ++n) {
                apply_h(o, ph + (size_t)(n - 1) * qs, y);
                cplx f = -I * h / (double)n;
                for (int i = 0; i < q; ++i) ph[(size_t)n * qs + i] = f * y[i];
            }
        }
        if (dL_dC) {   /* C(t_k) = sum_j conj(psi0_j) c(key_j)  =>  gbar_j += psi0_j w_k */
            cplx w = dL_dC[2 * k] + I * dL_dC[2 * k + 1];
            for (int j = 0; j < o->init.nrows; ++j) {
                int i = rs_find(&o->rows, rs_row(&o->init, j));
                if (i >= 0) gbar[i] += o->c0[j] * w;
            }
        }
        if (dL_dP) {   /* P_s(t_k) = sum_{i: site s} |c_i|^2  =>  gbar_i += 2 c_i dL/dP_s */
            const cplx* last_ph = phis + (size_t)base[ns - 1] * qs;
            int nl = R->sub_terms[ns - 1];
            for (int i = 0; i < q; ++i) {
                cplx c = 0.0;
                for (int n = 0; n <= nl; ++n) c += last_ph[(size_t)n * qs + i];
                gbar[i] += 2.0 * c * dL_dP[(size_t)k * N + rs_row(&o->rows, i)[0]];
            }
        }
        /* reverse recurrence, series by series from the last: gbar is the
         * cotangent of the series' output, mu ends as that of its input */
        for (int j = ns - 1; j >= 0; --j) {
            const cplx* ph = phis + (size_t)base[j] * qs;
            memcpy(mu, gbar, sizeof(cplx) * (size_t)q);
            for (int n = R->sub_terms[j]; n >= 1; --n) {
                cplx f = -I * h / (double)n;
                const cplx* phi_prev = ph + (size_t)(n - 1) * qs;
                for (int p = 0; p < P; ++p) {
                    apply_dh(o, p, phi_prev, y);
                    cplx sacc = 0.0;
                    for (int i = 0; i < q; ++i) sacc += conj(mu[i]) * (f * y[i]);
                    grad[p] += creal(sacc);
                }
                apply_h(o, mu, y);                     /* B_n^dag mu = (i h/n) H mu */
                for (int i = 0; i < q; ++i) mu[i] = gbar[i] + conj(f) * y[i];
            }
            if (j > 0) memcpy(gbar, mu, sizeof(cplx) * (size_t)q);
        }
        free(base);
        /* mu is now the cotangent of c'; scatter through the rescue map */
        cplx* prev = (cplx*)calloc((size_t)R->nprev + 1, sizeof(cplx));
        for (int i = 0; i < q; ++i)
            if (R->from[i] >= 0) prev[R->from[i]] += mu[i];
        free(gbar);
        gbar = prev;
        free(phis); free(y); free(mu);
    }
    free(gbar);
    rs_free(&o->rows);
    o->rows = live;
    free(o->c);
    o->c = live_c;
    o->ccap = live_ccap;
    or_build_hamiltonian(o, NULL, NULL, NULL, NULL);
    return rc;
}
