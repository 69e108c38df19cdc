/*
 * lbm_oracle.c - plain FP64 CPU oracle for the two lattice-Boltzmann Maxwell schemes compared in
 * arXiv 2309.08068: the Mendoza-Munoz model (MM, Section II) and the modified Hauser-Verhey model
 * (HV, Section III with the source term of eq. SourceTermHV).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product: only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it. The GPU library shares no code, header,
 * table or helper with it. Every step below is written in the paper's order and notation, in plain
 * loops, without blocking or fusion, so that it can be read against the paper line by line:
 *
 *   init  (Appendix B): f := f_eq(E, B, J = 0) at every cell, t := 0
 *   step  (Appendix B, loop body), for every cell x, iteration t (1-based):
 *     (i)   macroscopic moments          MM: eq. MacroscopicFieldsMiller   HV: eq. MacroscopicFieldsHV
 *     (ii)  external current J_ext(x, t) = sum over current sources of w(x) s(t)
 *     (iii) E and J                      MM: eqs. MacroscopicEMiller, MacorscopicCurrentMiller
 *                                        HV: E = D / eps, J = sigma E + J_ext (Appendix B note)
 *     (iv)  equilibria                   MM: eq. equilibriumsMiller        HV: eq. equilibriumHV
 *     (v)   BGK collision, tau = 1/2     MM: eq. CollisionMiller           HV: eq. CollisionmodifiedHV
 *     (vi)  imposed cells: f' := f_eq(E_imp(t), B_imp(t), J = 0)           (Appendix B "impose fields")
 *     (vii) advection f(x + v, t + 1) = f'(x, t), periodic on every axis
 *
 * Readings taken where the paper is silent or ambiguous:
 *   - MM units eps0 = 1, mu0 = 2 (Section II-A); H reported as B / (mu0 mu_r).
 *   - MM with both an ohmic sigma and an external current: E = (D'/eps_r - mu0 J_ext/(4 eps_r)) /
 *     (1 + mu0 sigma/(4 eps_r)), J = sigma E + J_ext; it reduces to each printed form.
 *   - MM rest populations: f_0^(0) collides as eq. CollisionMiller and feeds rho_c only; f_0^(1) has no
 *     collision rule in the paper and is carried unchanged.
 *   - HV units: eps0 * mu0 = 9 (vacuum speed 1/3, Section III-A); default eps0 = mu0 = 3.
 *   - Imposed cells keep the MM rest populations' collided values.
 *   - Source time argument: iteration t uses s(t); fields at time t use J_ext(t + 1).
 *
 * Memory layout: f[cell * q + k], cell = x + nx * (y + ny * z). Canonical population index k:
 *   MM (q = 50): k = r*24 + p*8 + (i-1)*2 + j  (r = 0 electric / 1 magnetic, plane p = 0..2,
 *                direction i = 1..4, j = 0..1);  k = 48 is f_0^(0), k = 49 is f_0^(1).
 *   HV (q = 36): k = r*18 + (i-1)*3 + c        (r = 0 electric vector e_i / 1 magnetic vector h_i,
 *                direction i = 1..6, component c = x, y, z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MM 0
#define OR_HV 1
#define OR_MAX_SOURCES 64

#define OR_FN_SIN 0
#define OR_FN_TABLE 1
#define OR_FN_CONST 2

#define OR_SRC_CURRENT 0
#define OR_SRC_IMPOSE 1

typedef struct {
    int kind;
    int64_t n;
    int64_t *cells;
    double *w; /* current sources: 3 weights per cell */
    double E0[3], B0[3]; /* imposed sources */
    int fn;
    double amp, period, phase;
    double *table;
    int64_t table_len;
} or_source;

typedef struct or_lattice {
    int model, nx, ny, nz, q;
    int64_t n;
    double eps0, mu0;
    double *eps_r, *mu_r, *sigma;
    double *f, *g;
    int64_t t;
    int nsrc;
    or_source src[OR_MAX_SOURCES];
    /* per-cell source scratch, valid at source cells only */
    double *jext, *eimp, *bimp;
    unsigned char *is_imposed;
    int nthreads;
    /* MM: velocity v[p][i-1], electric e[p][i-1][j], magnetic b[p][i-1][j] */
    double mm_v[3][4][3], mm_e[3][4][2][3], mm_b[3][4][2][3];
    /* HV: v[i-1] */
    double hv_v[6][3];
} or_lattice;

/* ------------------------------------------------------------------------------------------ */
/* Vector sets                                                                                */
/* ------------------------------------------------------------------------------------------ */

static double snap_half(double a) {
    /* The paper's trigonometric formulas give integers (v) or halves (e) up to rounding. */
    return nearbyint(2.0 * a) / 2.0;
}

static void cross(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* MM velocity set, eq. VelocitySetMiller, and electromagnetic vectors, eq. ElectromagneticVectorsMiller. */
static void build_mm_tables(or_lattice *L) {
    const double pi = 3.14159265358979323846;
    for (int p = 0; p < 3; ++p) {
        for (int i = 1; i <= 4; ++i) {
            double c = sqrt(2.0) * cos((2 * i - 1) * pi / 4.0);
            double s = sqrt(2.0) * sin((2 * i - 1) * pi / 4.0);
            double *v = L->mm_v[p][i - 1];
            if (p == 0) { v[0] = c; v[1] = s; v[2] = 0.0; }
            if (p == 1) { v[0] = c; v[1] = 0.0; v[2] = s; }
            if (p == 2) { v[0] = 0.0; v[1] = c; v[2] = s; }
            for (int a = 0; a < 3; ++a) v[a] = snap_half(v[a]);
        }
    }
    for (int p = 0; p < 3; ++p) {
        for (int i = 1; i <= 4; ++i) {
            int i0 = ((i + 2) % 4) + 1; /* e_{i0} = v_{[(i+2) mod 4]+1} / 2 */
            int i1 = (i % 4) + 1;       /* e_{i1} = v_{[i mod 4]+1} / 2 */
            for (int a = 0; a < 3; ++a) {
                L->mm_e[p][i - 1][0][a] = 0.5 * L->mm_v[p][i0 - 1][a];
                L->mm_e[p][i - 1][1][a] = 0.5 * L->mm_v[p][i1 - 1][a];
            }
            for (int j = 0; j < 2; ++j) cross(L->mm_v[p][i - 1], L->mm_e[p][i - 1][j], L->mm_b[p][i - 1][j]);
        }
    }
}

/* HV velocity set, Section III: v1 = +x, v2 = +y, v3 = -x, v4 = -y, v5 = -z, v6 = +z. */
static void build_hv_tables(or_lattice *L) {
    static const double v[6][3] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {0, 0, 1}};
    memcpy(L->hv_v, v, sizeof(v));
}

static int mm_k(int r, int p, int i, int j) { return r * 24 + p * 8 + (i - 1) * 2 + j; }
static int hv_k(int r, int i, int c) { return r * 18 + (i - 1) * 3 + c; }

/* ------------------------------------------------------------------------------------------ */
/* Sources                                                                                    */
/* ------------------------------------------------------------------------------------------ */

static double source_time_value(const or_source *s, int64_t t) {
    const double pi = 3.14159265358979323846;
    if (s->fn == OR_FN_SIN) return s->amp * sin(2.0 * pi * (double)t / s->period + s->phase);
    if (s->fn == OR_FN_TABLE) return (t >= 0 && t < s->table_len) ? s->amp * s->table[t] : 0.0;
    return s->amp; /* OR_FN_CONST */
}

/* Fill J_ext, E_imp, B_imp and the imposed flag at every source cell for time argument t. */
static void evaluate_sources(or_lattice *L, int64_t t) {
    for (int k = 0; k < L->nsrc; ++k) {
        const or_source *s = &L->src[k];
        for (int64_t m = 0; m < s->n; ++m) {
            int64_t x = s->cells[m];
            for (int a = 0; a < 3; ++a) {
                L->jext[3 * x + a] = 0.0;
                L->eimp[3 * x + a] = 0.0;
                L->bimp[3 * x + a] = 0.0;
            }
            L->is_imposed[x] = 0;
        }
    }
    for (int k = 0; k < L->nsrc; ++k) {
        const or_source *s = &L->src[k];
        double st = source_time_value(s, t);
        for (int64_t m = 0; m < s->n; ++m) {
            int64_t x = s->cells[m];
            if (s->kind == OR_SRC_CURRENT) {
                for (int a = 0; a < 3; ++a) L->jext[3 * x + a] += s->w[3 * m + a] * st;
            } else {
                for (int a = 0; a < 3; ++a) {
                    L->eimp[3 * x + a] += s->E0[a] * st;
                    L->bimp[3 * x + a] += s->B0[a] * st;
                }
                L->is_imposed[x] = 1;
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* MM model (Section II)                                                                      */
/* ------------------------------------------------------------------------------------------ */

/* Moments, eq. MacroscopicFieldsMiller: D' = sum f^(0) e, B = sum f^(1) b, rho_c = f_0^(0) + sum f^(0). */
static void mm_moments(const or_lattice *L, const double *f, double Dp[3], double B[3], double *rho) {
    Dp[0] = Dp[1] = Dp[2] = 0.0;
    B[0] = B[1] = B[2] = 0.0;
    *rho = f[48];
    for (int p = 0; p < 3; ++p)
        for (int i = 1; i <= 4; ++i)
            for (int j = 0; j < 2; ++j) {
                double f0 = f[mm_k(0, p, i, j)], f1 = f[mm_k(1, p, i, j)];
                for (int a = 0; a < 3; ++a) {
                    Dp[a] += f0 * L->mm_e[p][i - 1][j][a];
                    B[a] += f1 * L->mm_b[p][i - 1][j][a];
                }
                *rho += f0;
            }
}

/* E and J from D' with ohmic conductivity and an external current, eqs. MacroscopicEMiller and
 * MacorscopicCurrentMiller combined: E = E' - mu0 J/(4 eps_r), J = sigma E + J_ext, E' = D'/eps_r. */
static void mm_e_and_j(const or_lattice *L, int64_t x, const double Dp[3], const double Jext[3], double E[3],
                       double J[3]) {
    double er = L->eps_r[x], sg = L->sigma[x], mu0 = L->mu0;
    for (int a = 0; a < 3; ++a) {
        E[a] = (Dp[a] / er - mu0 * Jext[a] / (4.0 * er)) / (1.0 + mu0 * sg / (4.0 * er));
        J[a] = sg * E[a] + Jext[a];
    }
}

/* Equilibria, eq. equilibriumsMiller, for the 48 moving populations; out[48], out[49] untouched. */
static void mm_equilibrium(const or_lattice *L, int64_t x, const double E[3], const double B[3], const double J[3],
                           double *feq) {
    double er = L->eps_r[x], mr = L->mu_r[x];
    for (int p = 0; p < 3; ++p)
        for (int i = 1; i <= 4; ++i)
            for (int j = 0; j < 2; ++j) {
                const double *v = L->mm_v[p][i - 1], *e = L->mm_e[p][i - 1][j], *b = L->mm_b[p][i - 1][j];
                feq[mm_k(0, p, i, j)] = dot(v, J) / 16.0 + er / 4.0 * dot(E, e) + dot(B, b) / (8.0 * mr);
                feq[mm_k(1, p, i, j)] = dot(v, J) / 16.0 + dot(E, e) / 4.0 + dot(B, b) / 8.0;
            }
}

static void mm_collide(const or_lattice *L, int64_t x, const double *f, double *out) {
    static const double zero3[3] = {0.0, 0.0, 0.0};
    double Dp[3], B[3], rho, E[3], J[3], feq[50];
    const double *jext = L->jext ? &L->jext[3 * x] : zero3;
    mm_moments(L, f, Dp, B, &rho);                  /* (i)  */
    mm_e_and_j(L, x, Dp, jext, E, J);               /* (ii), (iii) */
    mm_equilibrium(L, x, E, B, J, feq);             /* (iv) */
    for (int k = 0; k < 48; ++k) out[k] = 2.0 * feq[k] - f[k]; /* (v) eq. CollisionMiller */
    out[48] = 2.0 * rho - f[48];                    /* f_0^(0)eq = rho_c */
    out[49] = f[49];                                /* f_0^(1): no rule in the paper, carried */
    if (L->is_imposed && L->is_imposed[x]) {        /* (vi) */
        mm_equilibrium(L, x, &L->eimp[3 * x], &L->bimp[3 * x], zero3, out);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Modified HV model (Section III)                                                            */
/* ------------------------------------------------------------------------------------------ */

/* Moments, eq. MacroscopicFieldsHV: D = sum e_i, B = sum h_i. */
static void hv_moments(const double *f, double D[3], double B[3]) {
    for (int a = 0; a < 3; ++a) {
        D[a] = 0.0;
        B[a] = 0.0;
        for (int i = 1; i <= 6; ++i) {
            D[a] += f[hv_k(0, i, a)];
            B[a] += f[hv_k(1, i, a)];
        }
    }
}

/* Equilibria, eq. equilibriumHV: e_i = (D - 3 v_i x B / mu) / 6, h_i = (B + 3 v_i x D / eps) / 6. */
static void hv_equilibrium(const or_lattice *L, int i, const double D[3], const double B[3], double eps, double mu,
                           double e_eq[3], double h_eq[3]) {
    double vxB[3], vxD[3];
    cross(L->hv_v[i - 1], B, vxB);
    cross(L->hv_v[i - 1], D, vxD);
    for (int a = 0; a < 3; ++a) {
        e_eq[a] = (D[a] - 3.0 * vxB[a] / mu) / 6.0;
        h_eq[a] = (B[a] + 3.0 * vxD[a] / eps) / 6.0;
    }
}

static void hv_collide(const or_lattice *L, int64_t x, const double *f, double *out) {
    static const double zero3[3] = {0.0, 0.0, 0.0};
    double eps = L->eps0 * L->eps_r[x], mu = L->mu0 * L->mu_r[x], sg = L->sigma[x];
    double D[3], B[3], E[3], J[3];
    const double *jext = L->jext ? &L->jext[3 * x] : zero3;
    hv_moments(f, D, B);                                   /* (i)  */
    for (int a = 0; a < 3; ++a) {                          /* (ii), (iii) */
        E[a] = D[a] / eps;
        J[a] = sg * E[a] + jext[a];
    }
    for (int i = 1; i <= 6; ++i) {
        double e_eq[3], h_eq[3], T[3];
        const double *v = L->hv_v[i - 1];
        hv_equilibrium(L, i, D, B, eps, mu, e_eq, h_eq);   /* (iv) */
        double jv = dot(J, v);                             /* eq. SourceTermHV: T_i = -(J.v_i) v_i / 2 */
        for (int a = 0; a < 3; ++a) T[a] = -0.5 * jv * v[a];
        for (int a = 0; a < 3; ++a) {                      /* (v) eqs. CollisionHV, CollisionmodifiedHV */
            out[hv_k(0, i, a)] = 2.0 * e_eq[a] - f[hv_k(0, i, a)] + T[a];
            out[hv_k(1, i, a)] = 2.0 * h_eq[a] - f[hv_k(1, i, a)];
        }
    }
    if (L->is_imposed && L->is_imposed[x]) {               /* (vi) */
        double Dimp[3];
        for (int a = 0; a < 3; ++a) Dimp[a] = eps * L->eimp[3 * x + a];
        for (int i = 1; i <= 6; ++i) {
            double e_eq[3], h_eq[3];
            hv_equilibrium(L, i, Dimp, &L->bimp[3 * x], eps, mu, e_eq, h_eq);
            for (int a = 0; a < 3; ++a) {
                out[hv_k(0, i, a)] = e_eq[a];
                out[hv_k(1, i, a)] = h_eq[a];
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Lattice bookkeeping                                                                        */
/* ------------------------------------------------------------------------------------------ */

static int64_t wrap(int64_t a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

static int64_t cell_index(const or_lattice *L, int64_t x, int64_t y, int64_t z) {
    return wrap(x, L->nx) + (int64_t)L->nx * (wrap(y, L->ny) + (int64_t)L->ny * wrap(z, L->nz));
}

/* Velocity of canonical population k (zero for rest populations). */
static void velocity_of(const or_lattice *L, int k, int v[3]) {
    v[0] = v[1] = v[2] = 0;
    if (L->model == OR_MM) {
        if (k >= 48) return;
        int p = (k % 24) / 8, i = (k % 8) / 2 + 1;
        for (int a = 0; a < 3; ++a) v[a] = (int)L->mm_v[p][i - 1][a];
    } else {
        int i = (k % 18) / 3 + 1;
        for (int a = 0; a < 3; ++a) v[a] = (int)L->hv_v[i - 1][a];
    }
}

int or_create(int model, int nx, int ny, int nz, const double *eps_r, const double *mu_r, const double *sigma,
              double eps0, double mu0, or_lattice **out) {
    if (!out || (model != OR_MM && model != OR_HV) || nx < 1 || ny < 1 || nz < 1) return -1;
    or_lattice *L = (or_lattice *)calloc(1, sizeof(or_lattice));
    if (!L) return -2;
    L->model = model;
    L->nx = nx;
    L->ny = ny;
    L->nz = nz;
    L->n = (int64_t)nx * ny * nz;
    L->q = model == OR_MM ? 50 : 36;
    if (model == OR_MM) {
        L->eps0 = eps0 > 0 ? eps0 : 1.0;
        L->mu0 = mu0 > 0 ? mu0 : 2.0;
        build_mm_tables(L);
    } else {
        L->eps0 = eps0 > 0 ? eps0 : 3.0;
        L->mu0 = mu0 > 0 ? mu0 : 3.0;
        build_hv_tables(L);
    }
    L->eps_r = (double *)malloc(sizeof(double) * L->n);
    L->mu_r = (double *)malloc(sizeof(double) * L->n);
    L->sigma = (double *)malloc(sizeof(double) * L->n);
    L->f = (double *)calloc((size_t)L->n * L->q, sizeof(double));
    L->g = (double *)calloc((size_t)L->n * L->q, sizeof(double));
    if (!L->eps_r || !L->mu_r || !L->sigma || !L->f || !L->g) {
        free(L->eps_r); free(L->mu_r); free(L->sigma); free(L->f); free(L->g); free(L);
        return -2;
    }
    for (int64_t x = 0; x < L->n; ++x) {
        L->eps_r[x] = eps_r ? eps_r[x] : 1.0;
        L->mu_r[x] = mu_r ? mu_r[x] : 1.0;
        L->sigma[x] = sigma ? sigma[x] : 0.0;
    }
    L->nthreads = 1;
    *out = L;
    return 0;
}

static void free_sources(or_lattice *L) {
    for (int k = 0; k < L->nsrc; ++k) {
        free(L->src[k].cells);
        free(L->src[k].w);
        free(L->src[k].table);
    }
    L->nsrc = 0;
    free(L->jext); free(L->eimp); free(L->bimp); free(L->is_imposed);
    L->jext = L->eimp = L->bimp = NULL;
    L->is_imposed = NULL;
}

void or_destroy(or_lattice *L) {
    if (!L) return;
    free_sources(L);
    free(L->eps_r); free(L->mu_r); free(L->sigma); free(L->f); free(L->g);
    free(L);
}

void or_set_threads(or_lattice *L, int nthreads) { L->nthreads = nthreads > 0 ? nthreads : 1; }
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}
int64_t or_time(const or_lattice *L) { return L->t; }
double or_eps0(const or_lattice *L) { return L->eps0; }
double or_mu0(const or_lattice *L) { return L->mu0; }

void or_clear_sources(or_lattice *L) { free_sources(L); }

/* kind: OR_SRC_CURRENT (w: 3 per cell) or OR_SRC_IMPOSE (E0, B0). fn: OR_FN_*. */
int or_add_source(or_lattice *L, int kind, int64_t n_cells, const int64_t *cells, const double *w, const double *E0,
                  const double *B0, int fn, double amp, double period, double phase, const double *table,
                  int64_t table_len) {
    if (L->nsrc >= OR_MAX_SOURCES || n_cells < 0 || (n_cells > 0 && !cells)) return -1;
    if (kind != OR_SRC_CURRENT && kind != OR_SRC_IMPOSE) return -1;
    if (kind == OR_SRC_CURRENT && n_cells > 0 && !w) return -1;
    if (kind == OR_SRC_IMPOSE && (!E0 || !B0)) return -1;
    if (fn == OR_FN_SIN && !(period != 0.0)) return -1;
    if (fn == OR_FN_TABLE && (table_len < 0 || (table_len > 0 && !table))) return -1;
    for (int64_t m = 0; m < n_cells; ++m)
        if (cells[m] < 0 || cells[m] >= L->n) return -1;
    if (!L->jext) {
        L->jext = (double *)calloc((size_t)3 * L->n, sizeof(double));
        L->eimp = (double *)calloc((size_t)3 * L->n, sizeof(double));
        L->bimp = (double *)calloc((size_t)3 * L->n, sizeof(double));
        L->is_imposed = (unsigned char *)calloc((size_t)L->n, 1);
        if (!L->jext || !L->eimp || !L->bimp || !L->is_imposed) return -2;
    }
    or_source *s = &L->src[L->nsrc];
    memset(s, 0, sizeof(*s));
    s->kind = kind;
    s->n = n_cells;
    s->cells = (int64_t *)malloc(sizeof(int64_t) * (n_cells > 0 ? n_cells : 1));
    memcpy(s->cells, cells, sizeof(int64_t) * n_cells);
    if (kind == OR_SRC_CURRENT) {
        s->w = (double *)malloc(sizeof(double) * 3 * (n_cells > 0 ? n_cells : 1));
        memcpy(s->w, w, sizeof(double) * 3 * n_cells);
    } else {
        memcpy(s->E0, E0, sizeof(s->E0));
        memcpy(s->B0, B0, sizeof(s->B0));
    }
    s->fn = fn;
    s->amp = amp;
    s->period = period;
    s->phase = phase;
    if (fn == OR_FN_TABLE && table_len > 0) {
        s->table = (double *)malloc(sizeof(double) * table_len);
        memcpy(s->table, table, sizeof(double) * table_len);
        s->table_len = table_len;
    }
    L->nsrc++;
    return 0;
}

/* Appendix B, first two lines: every population at its equilibrium for the given E, B and J = 0.
 * MM: D' = eps_r E (J = 0 in eq. MacroscopicEMiller); rho_c = 0 so both rest populations start at 0.
 * HV: D = eps0 eps_r E. E and B are component-major (3 x n). */
void or_init_fields(or_lattice *L, const double *E, const double *B) {
    static const double zero3[3] = {0.0, 0.0, 0.0};
    for (int64_t x = 0; x < L->n; ++x) {
        double Ex[3], Bx[3];
        for (int a = 0; a < 3; ++a) {
            Ex[a] = E[a * L->n + x];
            Bx[a] = B[a * L->n + x];
        }
        double *f = &L->f[x * L->q];
        if (L->model == OR_MM) {
            mm_equilibrium(L, x, Ex, Bx, zero3, f);
            f[48] = 0.0;
            f[49] = 0.0;
        } else {
            double eps = L->eps0 * L->eps_r[x], mu = L->mu0 * L->mu_r[x], D[3];
            for (int a = 0; a < 3; ++a) D[a] = eps * Ex[a];
            for (int i = 1; i <= 6; ++i) {
                double e_eq[3], h_eq[3];
                hv_equilibrium(L, i, D, Bx, eps, mu, e_eq, h_eq);
                for (int a = 0; a < 3; ++a) {
                    f[hv_k(0, i, a)] = e_eq[a];
                    f[hv_k(1, i, a)] = h_eq[a];
                }
            }
        }
    }
    L->t = 0;
}

/* One time step: collide every cell (steps i-vi) and advect (step vii) into g, then swap. */
static void one_step(or_lattice *L) {
    int64_t t_iter = L->t + 1;
    if (L->nsrc > 0) evaluate_sources(L, t_iter);
    const int q = L->q;
    int vel[50][3];
    for (int k = 0; k < q; ++k) velocity_of(L, k, vel[k]);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(L->nthreads)
#endif
    for (int z = 0; z < L->nz; ++z) {
        double out[50];
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                int64_t c = cell_index(L, x, y, z);
                const double *f = &L->f[c * q];
                if (L->model == OR_MM) mm_collide(L, c, f, out);
                else hv_collide(L, c, f, out);
                for (int k = 0; k < q; ++k) {
                    int64_t d = cell_index(L, x + vel[k][0], y + vel[k][1], z + vel[k][2]);
                    L->g[d * q + k] = out[k];
                }
            }
    }
    double *tmp = L->f;
    L->f = L->g;
    L->g = tmp;
    L->t = t_iter;
}

void or_step(or_lattice *L, int64_t n) {
    for (int64_t s = 0; s < n; ++s) one_step(L);
}

/* Fields at the current time t: moments of the stored populations, with the external current of
 * iteration t + 1 (the one the next collision will use). out = 15 x n, component-major, in the order
 * E, B, D, H, J. MM: D = eps0 eps_r E, H = B / (mu0 mu_r). HV: D, B moments, E = D/eps, H = B/mu. */
void or_fields(or_lattice *L, double *out) {
    static const double zero3[3] = {0.0, 0.0, 0.0};
    if (L->nsrc > 0) evaluate_sources(L, L->t + 1);
    const int64_t n = L->n;
    for (int64_t x = 0; x < n; ++x) {
        const double *f = &L->f[x * L->q];
        const double *jext = L->jext ? &L->jext[3 * x] : zero3;
        double E[3], B[3], D[3], H[3], J[3];
        if (L->model == OR_MM) {
            double Dp[3], rho;
            mm_moments(L, f, Dp, B, &rho);
            mm_e_and_j(L, x, Dp, jext, E, J);
            for (int a = 0; a < 3; ++a) {
                D[a] = L->eps0 * L->eps_r[x] * E[a];
                H[a] = B[a] / (L->mu0 * L->mu_r[x]);
            }
        } else {
            double eps = L->eps0 * L->eps_r[x], mu = L->mu0 * L->mu_r[x];
            hv_moments(f, D, B);
            for (int a = 0; a < 3; ++a) {
                E[a] = D[a] / eps;
                J[a] = L->sigma[x] * E[a] + jext[a];
                H[a] = B[a] / mu;
            }
        }
        for (int a = 0; a < 3; ++a) {
            out[(0 + a) * n + x] = E[a];
            out[(3 + a) * n + x] = B[a];
            out[(6 + a) * n + x] = D[a];
            out[(9 + a) * n + x] = H[a];
            out[(12 + a) * n + x] = J[a];
        }
    }
}

/* MM charge density rho_c per cell (eq. MacroscopicFieldsMiller); zero for HV. */
void or_charge(const or_lattice *L, double *out) {
    for (int64_t x = 0; x < L->n; ++x) {
        if (L->model != OR_MM) {
            out[x] = 0.0;
            continue;
        }
        double Dp[3], B[3], rho;
        mm_moments(L, &L->f[x * L->q], Dp, B, &rho);
        out[x] = rho;
    }
}

/* Populations in canonical component-major layout out[k * n + cell]. */
void or_get_populations(const or_lattice *L, double *out) {
    for (int64_t x = 0; x < L->n; ++x)
        for (int k = 0; k < L->q; ++k) out[(int64_t)k * L->n + x] = L->f[x * L->q + k];
}

void or_set_populations(or_lattice *L, const double *in, int64_t t) {
    for (int64_t x = 0; x < L->n; ++x)
        for (int k = 0; k < L->q; ++k) L->f[x * L->q + k] = in[(int64_t)k * L->n + x];
    L->t = t;
}

/* Vector tables as the oracle built them: MM v (12 x 3, index p*4 + i-1), e and b (24 x 3, index
 * (p*4 + i-1)*2 + j); HV v (6 x 3). */
void or_tables(const or_lattice *L, double *v, double *e, double *b) {
    if (L->model == OR_MM) {
        for (int p = 0; p < 3; ++p)
            for (int i = 0; i < 4; ++i)
                for (int a = 0; a < 3; ++a) {
                    v[(p * 4 + i) * 3 + a] = L->mm_v[p][i][a];
                    for (int j = 0; j < 2; ++j) {
                        e[((p * 4 + i) * 2 + j) * 3 + a] = L->mm_e[p][i][j][a];
                        b[((p * 4 + i) * 2 + j) * 3 + a] = L->mm_b[p][i][j][a];
                    }
                }
    } else {
        for (int i = 0; i < 6; ++i)
            for (int a = 0; a < 3; ++a) v[i * 3 + a] = L->hv_v[i][a];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint of one time step (for gradients of a loss with respect to eps_r and sigma)           */
/* ------------------------------------------------------------------------------------------ */
/*
 * One forward iteration maps the pre-collision populations f^n to f^{n+1}: collide every cell
 * (affine in its own populations), then advect f^{n+1}(x + v_k)[k] = f'(x)[k]. Given
 * g_next = dL/df^{n+1} (canonical layout), or_adjoint_step returns g_out = dL/df^n through this step
 * and adds dL/d eps_r and dL/d sigma of every cell.
 *
 * The transpose is taken by probing the oracle's own collision, not by a separate derivation:
 *   - the adjoint of the post-collision values of cell x is g_next(x + v_k)[k] (advection reversed);
 *   - column k of the collision's Jacobian is collide(unit k) - collide(0), so
 *     g_out(x)[k] = sum_m gp[m] * (collide(unit k)[m] - collide(0)[m]);
 *   - d collide / d eps_r and d collide / d sigma at f^n(x) are central differences in double
 *     precision (step 1e-6 relative), contracted with gp.
 * iter is the forward iteration number (its sources are s(iter)).
 */
static void collide_at(or_lattice *L, int64_t x, const double *f, double *out) {
    if (L->model == OR_MM) mm_collide(L, x, f, out);
    else hv_collide(L, x, f, out);
}

void or_adjoint_step(or_lattice *L, int64_t iter, const double *g_next, const double *f_n, double *g_out,
                     double *grad_eps_r, double *grad_sigma) {
    const int q = L->q;
    const int64_t n = L->n;
    int vel[50][3];
    for (int k = 0; k < q; ++k) velocity_of(L, k, vel[k]);
    if (L->nsrc > 0) evaluate_sources(L, iter);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(L->nthreads)
#endif
    for (int z = 0; z < L->nz; ++z) {
        double gp[50], f[50], unit[50], base[50], probe[50], plus[50], minus[50];
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                int64_t c = cell_index(L, x, y, z);
                for (int k = 0; k < q; ++k) {
                    int64_t d = cell_index(L, x + vel[k][0], y + vel[k][1], z + vel[k][2]);
                    gp[k] = g_next[(int64_t)k * n + d];
                    f[k] = f_n[(int64_t)k * n + c];
                    unit[k] = 0.0;
                }
                collide_at(L, c, unit, base);
                for (int k = 0; k < q; ++k) {
                    unit[k] = 1.0;
                    collide_at(L, c, unit, probe);
                    unit[k] = 0.0;
                    double s = 0.0;
                    for (int m = 0; m < q; ++m) s += gp[m] * (probe[m] - base[m]);
                    g_out[(int64_t)k * n + c] = s;
                }
                double *param[2] = {&L->eps_r[c], &L->sigma[c]};
                double *grad[2] = {grad_eps_r, grad_sigma};
                for (int p = 0; p < 2; ++p) {
                    if (!grad[p]) continue;
                    double v0 = *param[p];
                    double h = 1e-6 * (fabs(v0) > 1e-3 ? fabs(v0) : 1e-3);
                    *param[p] = v0 + h;
                    collide_at(L, c, f, plus);
                    *param[p] = v0 - h;
                    collide_at(L, c, f, minus);
                    *param[p] = v0;
                    double s = 0.0;
                    for (int m = 0; m < q; ++m) s += gp[m] * (plus[m] - minus[m]) / (2.0 * h);
                    grad[p][c] += s;
                }
            }
    }
}

/* Loss term of one time: L_t = sum over the cells of plane (axis, index) of |E(f, t)|^2, E as in
 * or_fields (external current of iteration t + 1). Returns L_t; adds dL_t/df to g (canonical) and
 * dL_t/d eps_r, dL_t/d sigma to the gradients. The derivatives are probed like or_adjoint_step: E is
 * affine in f, so dE/df_k = E(unit k) - E(0); parameters by central differences. */
static void fields_at(or_lattice *L, int64_t x, const double *f, double E[3]) {
    static const double zero3[3] = {0.0, 0.0, 0.0};
    const double *jext = L->jext ? &L->jext[3 * x] : zero3;
    if (L->model == OR_MM) {
        double Dp[3], B[3], rho, J[3];
        mm_moments(L, f, Dp, B, &rho);
        mm_e_and_j(L, x, Dp, jext, E, J);
    } else {
        double D[3], B[3], eps = L->eps0 * L->eps_r[x];
        hv_moments(f, D, B);
        for (int a = 0; a < 3; ++a) E[a] = D[a] / eps;
    }
}

double or_plane_loss(or_lattice *L, int64_t t, const double *f_t, int axis, int index, double *g, double *grad_eps_r,
                     double *grad_sigma) {
    const int q = L->q;
    const int64_t n = L->n;
    if (L->nsrc > 0) evaluate_sources(L, t + 1);
    double loss = 0.0;
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                int coord = axis == 0 ? x : (axis == 1 ? y : z);
                if (coord != index) continue;
                int64_t c = cell_index(L, x, y, z);
                double f[50], unit[50], E[3], E0[3], Ek[3];
                for (int k = 0; k < q; ++k) {
                    f[k] = f_t[(int64_t)k * n + c];
                    unit[k] = 0.0;
                }
                fields_at(L, c, f, E);
                loss += E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
                if (g) {
                    fields_at(L, c, unit, E0);
                    for (int k = 0; k < q; ++k) {
                        unit[k] = 1.0;
                        fields_at(L, c, unit, Ek);
                        unit[k] = 0.0;
                        double s = 0.0;
                        for (int a = 0; a < 3; ++a) s += 2.0 * E[a] * (Ek[a] - E0[a]);
                        g[(int64_t)k * n + c] += s;
                    }
                }
                double *param[2] = {&L->eps_r[c], &L->sigma[c]};
                double *grad[2] = {grad_eps_r, grad_sigma};
                for (int p = 0; p < 2; ++p) {
                    if (!grad[p]) continue;
                    double v0 = *param[p], Ep[3], Em[3];
                    double h = 1e-6 * (fabs(v0) > 1e-3 ? fabs(v0) : 1e-3);
                    *param[p] = v0 + h;
                    fields_at(L, c, f, Ep);
                    *param[p] = v0 - h;
                    fields_at(L, c, f, Em);
                    *param[p] = v0;
                    double s = 0.0;
                    for (int a = 0; a < 3; ++a) s += 2.0 * E[a] * (Ep[a] - Em[a]) / (2.0 * h);
                    grad[p][c] += s;
                }
            }
    return loss;
}
