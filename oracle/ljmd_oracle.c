/*
 * Plain FP64 CPU oracle for truncated Lennard-Jones molecular dynamics.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only the test suite, the
 * package's smoke check and the benchmark's CPU-baseline leg may load this
 * library. It shares no code with the CUDA path.
 *
 * It follows Watanabe, Suzuki and Ito, "Huge-scale Molecular Dynamics
 * Simulation of Multibubble Nuclei" (arXiv:1210.3450):
 *   - Sec. 2.1, Eq. 1: V(r) = 4[r^-12 - r^-6 + c2 r^2 + c0] for r < rc, with
 *     c2, c0 chosen so that V(rc) = V'(rc) = 0 (reduced units).
 *   - Sec. 2.1: grid (linked-list) cell search, bookkeeping (Verlet) list with a
 *     margin, list validity checked every step.
 *   - Sec. 2.1 / Fig. 1: pair list stored as key pointer + sorted partner list.
 *   - Sec. 3.3 / Algorithm 1: full list (no Newton's third law); per-pair
 *     force factor (24 r^6 - 48) / r^14 + 8 c2 times the separation vector.
 *   - Sec. 3.2 / Sec. 4.1: second-order symplectic integration (read as
 *     velocity Verlet, unit mass).
 *
 * Readings of points the paper leaves open (all stated again where used):
 *   - the list-validity check rebuilds when twice the largest minimum-image
 *     displacement since the last build reaches the skin;
 *   - cutoff and list radius are strict (r^2 < rc^2, r^2 < rl^2);
 *   - temperature is 2 KE / (3 (N - 1)); pressure is (2 KE + W) / (3 V).
 *
 * Compile with -O2 -ffp-contract=off: every product and sum below is rounded
 * on its own, in the order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------- Eq. 1 */

/* Coefficients of Eq. 1. V(rc) = 0 and V'(rc) = 0 give
 *   -12 rc^-13 + 6 rc^-7 + 2 c2 rc = 0  ->  c2 = 6 rc^-14 - 3 rc^-8
 *   rc^-12 - rc^-6 + c2 rc^2 + c0 = 0   ->  c0 = 4 rc^-6 - 7 rc^-12      */
ORC_API void orc_lj_coeffs(double rc, double* c2, double* c0) {
    double rc2 = rc * rc;
    double rc6 = rc2 * rc2 * rc2;
    double rc8 = rc6 * rc2;
    double rc12 = rc6 * rc6;
    double rc14 = rc12 * rc2;
    *c2 = 6.0 / rc14 - 3.0 / rc8;
    *c0 = 4.0 / rc6 - 7.0 / rc12;
}

/* V(r) of Eq. 1 for one pair at squared distance r2 (0 at or beyond rc). */
ORC_API double orc_pair_energy(double r2, double rc2, double c2, double c0) {
    if (!(r2 < rc2)) return 0.0;
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    return 4.0 * (ir6 * ir6 - ir6 + c2 * r2 + c0);
}

/* Force factor g(r) with F_i = g(r) (x_j - x_i): g = V'(r) / r
 *   = 24 r^-8 - 48 r^-14 + 8 c2  (the bracket of Algorithm 1 without dt). */
ORC_API double orc_pair_force_factor(double r2, double rc2, double c2) {
    if (!(r2 < rc2)) return 0.0;
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double ir8 = ir6 * ir2;
    double ir14 = ir8 * ir6;
    return 24.0 * ir8 - 48.0 * ir14 + 8.0 * c2;
}

/* Pair virial -r V'(r) = 48 r^-12 - 24 r^-6 - 8 c2 r^2. */
ORC_API double orc_pair_virial(double r2, double rc2, double c2) {
    if (!(r2 < rc2)) return 0.0;
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    return 48.0 * ir6 * ir6 - 24.0 * ir6 - 8.0 * c2 * r2;
}

/* ------------------------------------ reciprocal approximation (Sec. 3.3) */

/* Approximate reciprocal of r^2 standing in for SPARC64 frcpad: r^2 rounded to
 * float, its correctly rounded float reciprocal, the mantissa truncated to
 * `bits` bits (bits = 8 gives a relative error below 1/256 as Eq. 2 states;
 * bits >= 23 keeps the float value). */
static double approx_rcp(double r2, int bits) {
    float f = (float)r2;
    float y = 1.0f / f;
    if (bits < 23) {
        uint32_t u;
        memcpy(&u, &y, sizeof(u));
        u &= ~((1u << (23 - bits)) - 1u);
        memcpy(&y, &u, sizeof(u));
    }
    return (double)y;
}

/* Force factor of Algorithm 1 with r^-8 and r^-14 built from the approximate
 * reciprocal y of r^2 (Sec. 3.3): uncorrected y^4 and y^7, or corrected by
 * Eqs. 2-7: r^-8 ~ y^4 (5 - 4 y r^2), r^-14 ~ y^7 (8 - 7 y r^2). */
ORC_API double orc_pair_force_factor_rcp(double r2, double rc2, double c2, int bits, int corr) {
    if (!(r2 < rc2)) return 0.0;
    double y = approx_rcp(r2, bits);
    double y2 = y * y;
    double y4 = y2 * y2;
    double y7 = y4 * y2 * y;
    double ir8 = y4, ir14 = y7;
    if (corr) {
        double e = y * r2;
        ir8 = y4 * (5.0 - 4.0 * e);
        ir14 = y7 * (8.0 - 7.0 * e);
    }
    return 24.0 * ir8 - 48.0 * ir14 + 8.0 * c2;
}

/* ------------------------------------------------------- periodic box */

/* Minimum image of one separation component: d - L * nearbyint(d / L). */
static double min_image(double d, double box) { return d - box * nearbyint(d / box); }

/* Squared minimum-image distance from i to j, summed as (dx^2 + dy^2) + dz^2. */
static double dist2(const double* x, int64_t i, int64_t j, double box, double* dx, double* dy,
                    double* dz) {
    double ax = min_image(x[3 * j + 0] - x[3 * i + 0], box);
    double ay = min_image(x[3 * j + 1] - x[3 * i + 1], box);
    double az = min_image(x[3 * j + 2] - x[3 * i + 2], box);
    if (dx) { *dx = ax; *dy = ay; *dz = az; }
    return (ax * ax + ay * ay) + az * az;
}

/* Wrap one coordinate into [0, L): x - L floor(x / L), then fix the cases where
 * rounding leaves it at L or just below 0. */
static double wrap1(double x, double box) {
    double w = x - box * floor(x / box);
    if (w < 0.0) w = w + box;
    if (w >= box) w = w - box;
    if (w < 0.0 || w >= box) w = 0.0;
    return w;
}

ORC_API void orc_wrap(int64_t n, double box, double* x) {
    for (int64_t k = 0; k < 3 * n; ++k) x[k] = wrap1(x[k], box);
}

/* --------------------------------------------------- cell (grid) method */

/* Cells per axis: floor(L / rl), lowered by one when the cell side L / nc is not
 * clearly larger than rl (so rounding of x nc / L can never put a partner within
 * rl two cells away). The search uses cells only when the result is at least 3
 * (otherwise every pair is a candidate). */
ORC_API int orc_cells_per_axis(double box, double rl) {
    int nc = (int)floor(box / rl);
    if (nc >= 1 && box / nc < rl * (1.0 + 1e-9)) nc -= 1;
    return nc;
}

/* Linear cell of each particle: c_a = min(floor(x_a * nc / L), nc - 1),
 * index = cx + nc (cy + nc cz). Positions must already lie in [0, L). */
ORC_API void orc_cell_index(int64_t n, double box, int nc, const double* x, int32_t* cell) {
    double inv_cs = (double)nc / box;
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor(x[3 * i + a] * inv_cs);
            if (k > nc - 1) k = nc - 1;
            if (k < 0) k = 0;
            c[a] = k;
        }
        cell[i] = c[0] + nc * (c[1] + nc * c[2]);
    }
}

static int cmp_i32(const void* a, const void* b) {
    int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
    return (u > v) - (u < v);
}

/* Full pair list (both (i,j) and (j,i)): partners j != i with minimum-image
 * r^2 < rl^2, partners of i sorted ascending, stored as start[n+1] and
 * partners[...] (the key-pointer / sorted-list format of Fig. 1).
 * use_cells = 0 tests every pair (brute force); 1 uses the cell method when
 * there are at least 3 cells per axis. Returns the number of entries, or
 * -(needed) if cap is too small (nothing beyond cap is written). */
static int64_t build_list(int64_t n, double box, double rl, const double* x, int use_cells,
                          int64_t* start, int32_t* partners, int64_t cap) {
    double rl2 = rl * rl;
    int nc = orc_cells_per_axis(box, rl);
    int64_t total = 0;
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* cell = NULL;
    int64_t* head = NULL;
    int64_t* next = NULL;
    if (use_cells && nc >= 3) {
        int64_t ncell = (int64_t)nc * nc * nc;
        cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
        next = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        orc_cell_index(n, box, nc, x, cell);
        for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
        for (int64_t i = n - 1; i >= 0; --i) { next[i] = head[cell[i]]; head[cell[i]] = i; }
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t m = 0;
        if (cell) {
            int ci = cell[i];
            int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
            for (int oz = -1; oz <= 1; ++oz)
                for (int oy = -1; oy <= 1; ++oy)
                    for (int ox = -1; ox <= 1; ++ox) {
                        int nx = (cx + ox + nc) % nc, ny = (cy + oy + nc) % nc,
                            nz = (cz + oz + nc) % nc;
                        for (int64_t j = head[nx + nc * (ny + nc * nz)]; j >= 0; j = next[j]) {
                            if (j == i) continue;
                            if (dist2(x, i, j, box, 0, 0, 0) < rl2) cand[m++] = (int32_t)j;
                        }
                    }
        } else {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                if (dist2(x, i, j, box, 0, 0, 0) < rl2) cand[m++] = (int32_t)j;
            }
        }
        qsort(cand, (size_t)m, sizeof(int32_t), cmp_i32);
        start[i] = total;
        for (int64_t k = 0; k < m; ++k) {
            if (total + k < cap) partners[total + k] = cand[k];
        }
        total += m;
    }
    start[n] = total;
    free(cand);
    free(cell);
    free(head);
    free(next);
    return total <= cap ? total : -total;
}

ORC_API int64_t orc_build_list(int64_t n, double box, double rl, const double* x,
                               int64_t* start, int32_t* partners, int64_t cap) {
    return build_list(n, box, rl, x, 1, start, partners, cap);
}

ORC_API int64_t orc_build_list_brute(int64_t n, double box, double rl, const double* x,
                                     int64_t* start, int32_t* partners, int64_t cap) {
    return build_list(n, box, rl, x, 0, start, partners, cap);
}

/* ------------------------------------------------------------- forces */

/* F_i = sum over listed partners j with r < rc of g(r) (x_j - x_i), in list order
 * (ascending j). Newton's third law is not used (Sec. 3.3). */
ORC_API void orc_forces_list(int64_t n, double box, double rc, double c2, const double* x,
                             const int64_t* start, const int32_t* partners, double* f) {
    double rc2 = rc * rc;
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            double dx, dy, dz;
            double r2 = dist2(x, i, partners[k], box, &dx, &dy, &dz);
            double g = orc_pair_force_factor(r2, rc2, c2);
            fx += g * dx;
            fy += g * dy;
            fz += g * dz;
        }
        f[3 * i + 0] = fx;
        f[3 * i + 1] = fy;
        f[3 * i + 2] = fz;
    }
}

/* Forces with Newton's third law (Sec. 2.1: each pair once, i < j, the key particle's
 * sum gets +g r and the partner's -g r), taking from the full list only the partners
 * j > i, in list order. */
ORC_API void orc_forces_half(int64_t n, double box, double rc, double c2, const double* x,
                             const int64_t* start, const int32_t* partners, double* f) {
    double rc2 = rc * rc;
    for (int64_t k = 0; k < 3 * n; ++k) f[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = partners[k];
            if (j <= i) continue;
            double dx, dy, dz;
            double r2 = dist2(x, i, j, box, &dx, &dy, &dz);
            double g = orc_pair_force_factor(r2, rc2, c2);
            f[3 * i + 0] += g * dx;
            f[3 * i + 1] += g * dy;
            f[3 * i + 2] += g * dz;
            f[3 * j + 0] -= g * dx;
            f[3 * j + 1] -= g * dy;
            f[3 * j + 2] -= g * dz;
        }
    }
}

/* Forces over the list with the approximate-reciprocal force factor. */
ORC_API void orc_forces_list_rcp(int64_t n, double box, double rc, double c2, const double* x,
                                 const int64_t* start, const int32_t* partners, int bits, int corr,
                                 double* f) {
    double rc2 = rc * rc;
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            double dx, dy, dz;
            double r2 = dist2(x, i, partners[k], box, &dx, &dy, &dz);
            double g = orc_pair_force_factor_rcp(r2, rc2, c2, bits, corr);
            fx += g * dx;
            fy += g * dy;
            fz += g * dz;
        }
        f[3 * i + 0] = fx;
        f[3 * i + 1] = fy;
        f[3 * i + 2] = fz;
    }
}

/* Force on particle i by direct summation over all j != i (no list), j ascending. */
ORC_API void orc_force_on(int64_t n, double box, double rc, double c2, const double* x,
                          int64_t i, double* f3) {
    double rc2 = rc * rc;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx, dy, dz;
        double r2 = dist2(x, i, j, box, &dx, &dy, &dz);
        double g = orc_pair_force_factor(r2, rc2, c2);
        fx += g * dx;
        fy += g * dy;
        fz += g * dz;
    }
    f3[0] = fx;
    f3[1] = fy;
    f3[2] = fz;
}

ORC_API void orc_forces_brute(int64_t n, double box, double rc, double c2, const double* x,
                              double* f) {
    for (int64_t i = 0; i < n; ++i) orc_force_on(n, box, rc, c2, x, i, f + 3 * i);
}

/* -------------------------------------------------------- observables */

/* out[0] = PE = 1/2 sum_i sum_{j in list(i)} V(r)  (full list counts each pair twice)
 * out[1] = W  = 1/2 sum_i sum_j (-r V'(r))
 * out[2] = KE = 1/2 sum_i |v_i|^2
 * out[3] = T  = 2 KE / (3 (N - 1))
 * out[4] = P  = (2 KE + W) / (3 L^3)
 * Sums run over i ascending, then the list of i in order. */
ORC_API void orc_observables_list(int64_t n, double box, double rc, double c2, double c0,
                                  const double* x, const double* v, const int64_t* start,
                                  const int32_t* partners, double* out) {
    double rc2 = rc * rc;
    double pe = 0.0, w = 0.0, ke = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            double r2 = dist2(x, i, partners[k], box, 0, 0, 0);
            pe += orc_pair_energy(r2, rc2, c2, c0);
            w += orc_pair_virial(r2, rc2, c2);
        }
    }
    pe *= 0.5;
    w *= 0.5;
    for (int64_t k = 0; k < 3 * n; ++k) ke += v[k] * v[k];
    ke *= 0.5;
    out[0] = pe;
    out[1] = w;
    out[2] = ke;
    out[3] = n > 1 ? 2.0 * ke / (3.0 * (double)(n - 1)) : 0.0;
    out[4] = (2.0 * ke + w) / (3.0 * box * box * box);
}

/* --------------------------------------------------------- integrator */

typedef struct {
    int64_t n;
    double box, rc, skin, rl, c2, c0;
    double* x_ref;    /* positions at the last list build */
    int64_t* start;
    int32_t* partners;
    int64_t cap;
    int64_t rebuilds;
} orc_list_state;

static int list_rebuild(orc_list_state* s, const double* x) {
    for (;;) {
        int64_t got = orc_build_list(s->n, s->box, s->rl, x, s->start, s->partners, s->cap);
        if (got >= 0) break;
        free(s->partners);
        s->cap = -got + s->n;
        s->partners = (int32_t*)malloc(sizeof(int32_t) * (size_t)s->cap);
        if (!s->partners) return -1;
    }
    memcpy(s->x_ref, x, sizeof(double) * 3 * (size_t)s->n);
    s->rebuilds += 1;
    return 0;
}

/* Largest minimum-image displacement since the last build (exact FP64 max). */
static double max_displacement(const orc_list_state* s, const double* x) {
    double m2 = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
        double dx = min_image(x[3 * i + 0] - s->x_ref[3 * i + 0], s->box);
        double dy = min_image(x[3 * i + 1] - s->x_ref[3 * i + 1], s->box);
        double dz = min_image(x[3 * i + 2] - s->x_ref[3 * i + 2], s->box);
        double d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 > m2) m2 = d2;
    }
    return sqrt(m2);
}

/* Velocity Verlet (kick 1/2, drift, kick 1/2; unit mass) for nsteps steps, in
 * place on x (n*3, wrapped into [0, L) on entry) and v (n*3). The list is
 * built at the start and rebuilt after a drift whenever 2 * d_max >= skin.
 * If trace is not NULL it receives E = KE + PE at step 0 and after every
 * trace_every steps (1 + nsteps / trace_every entries).
 * Returns 0, or -1 on allocation failure. *rebuilds gets the number of builds
 * (including the initial one). */
static void forces_mode(const orc_list_state* s, const double* x, int rcp_bits, int rcp_corr,
                        double* f) {
    if (rcp_bits < 0)
        orc_forces_list(s->n, s->box, s->rc, s->c2, x, s->start, s->partners, f);
    else
        orc_forces_list_rcp(s->n, s->box, s->rc, s->c2, x, s->start, s->partners, rcp_bits,
                            rcp_corr, f);
}

/* As orc_run, with the approximate-reciprocal force factor when rcp_bits >= 0 and the
 * list validity rule `rule`: 0 displacement (2 d_max >= skin), 1 velocity bound (the DUTC
 * check of Sec. 2.1: a margin equal to the skin after each build shrinks by
 * 2 v_max dt per step, v_max the largest speed used in the drift; rebuild when the margin
 * is no longer positive). */
ORC_API int orc_run_rule(int64_t n, double box, double rc, double skin, double* x, double* v,
                         int64_t nsteps, double dt, int64_t* rebuilds, double* trace,
                         int64_t trace_every, int rcp_bits, int rcp_corr, int rule);

ORC_API int orc_run(int64_t n, double box, double rc, double skin, double* x, double* v,
                    int64_t nsteps, double dt, int64_t* rebuilds, double* trace,
                    int64_t trace_every) {
    return orc_run_rule(n, box, rc, skin, x, v, nsteps, dt, rebuilds, trace, trace_every, -1, 0, 0);
}

ORC_API int orc_run_mode(int64_t n, double box, double rc, double skin, double* x, double* v,
                         int64_t nsteps, double dt, int64_t* rebuilds, double* trace,
                         int64_t trace_every, int rcp_bits, int rcp_corr) {
    return orc_run_rule(n, box, rc, skin, x, v, nsteps, dt, rebuilds, trace, trace_every, rcp_bits,
                        rcp_corr, 0);
}

/* Largest speed |v_i| = sqrt((vx vx + vy vy) + vz vz). */
static double max_speed(int64_t n, const double* v) {
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s2 = (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1]) + v[3 * i + 2] * v[3 * i + 2];
        if (s2 > m) m = s2;
    }
    return sqrt(m);
}

ORC_API int orc_run_rule(int64_t n, double box, double rc, double skin, double* x, double* v,
                         int64_t nsteps, double dt, int64_t* rebuilds, double* trace,
                         int64_t trace_every, int rcp_bits, int rcp_corr, int rule) {
    orc_list_state s;
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.box = box;
    s.rc = rc;
    s.skin = skin;
    s.rl = rc + skin;
    orc_lj_coeffs(rc, &s.c2, &s.c0);
    s.cap = n * 128 + 64;
    s.partners = (int32_t*)malloc(sizeof(int32_t) * (size_t)s.cap);
    s.start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    s.x_ref = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    int rc_ = 0;
    if (!s.partners || !s.start || !s.x_ref || !f) { rc_ = -1; goto done; }
    orc_wrap(n, box, x);
    if (list_rebuild(&s, x)) { rc_ = -1; goto done; }
    forces_mode(&s, x, rcp_bits, rcp_corr, f);
    double hdt = 0.5 * dt;
    int64_t ti = 0;
    if (trace) {
        double o[5];
        orc_observables_list(n, box, rc, s.c2, s.c0, x, v, s.start, s.partners, o);
        trace[ti++] = o[0] + o[2];
    }
    double margin = skin;
    for (int64_t step = 1; step <= nsteps; ++step) {
        for (int64_t k = 0; k < 3 * n; ++k) v[k] = v[k] + hdt * f[k];
        for (int64_t k = 0; k < 3 * n; ++k) x[k] = wrap1(x[k] + dt * v[k], box);
        int rebuild_now;
        if (rule == 1) {
            margin = margin - (2.0 * max_speed(n, v)) * dt;
            rebuild_now = !(margin > 0.0);
        } else {
            rebuild_now = 2.0 * max_displacement(&s, x) >= skin;
        }
        if (rebuild_now) {
            if (list_rebuild(&s, x)) { rc_ = -1; goto done; }
            margin = skin;
        }
        forces_mode(&s, x, rcp_bits, rcp_corr, f);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] = v[k] + hdt * f[k];
        if (trace && trace_every > 0 && step % trace_every == 0) {
            double o[5];
            orc_observables_list(n, box, rc, s.c2, s.c0, x, v, s.start, s.partners, o);
            trace[ti++] = o[0] + o[2];
        }
    }
done:
    if (rebuilds) *rebuilds = s.rebuilds;
    free(s.partners);
    free(s.start);
    free(s.x_ref);
    free(f);
    return rc_;
}

/* ------------------------------------------------ bubbles (Sec. 4.2) */

/* Particles per subcell of the grid with ns subcells per axis (side L / ns):
 * c_a = min(floor(x_a (ns / L)), ns - 1), index cx + ns (cy + ns cz); positions in [0, L). */
ORC_API void orc_subcell_counts(int64_t n, double box, int ns, const double* x, int32_t* counts) {
    double inv = (double)ns / box;
    int64_t ncell = (int64_t)ns * ns * ns;
    for (int64_t c = 0; c < ncell; ++c) counts[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor(x[3 * i + a] * inv);
            if (k > ns - 1) k = ns - 1;
            if (k < 0) k = 0;
            c[a] = k;
        }
        counts[c[0] + ns * (c[1] + ns * c[2])] += 1;
    }
}

/* Site percolation on the periodic simple cubic lattice (Sec. 4.2): subcells with
 * gas[c] != 0 that share a face belong to the same cluster. Flood fill (breadth
 * first) from every unlabelled gas cell in index order; label[c] = smallest index
 * of c's cluster, -1 for non-gas cells. Returns the number of clusters. */
ORC_API int64_t orc_clusters(int ns, const uint8_t* gas, int32_t* label) {
    int64_t ncell = (int64_t)ns * ns * ns;
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ncell > 0 ? ncell : 1));
    int64_t nclusters = 0;
    for (int64_t c = 0; c < ncell; ++c) label[c] = -1;
    for (int64_t c0 = 0; c0 < ncell; ++c0) {
        if (!gas[c0] || label[c0] >= 0) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)c0;
        label[c0] = (int32_t)c0;
        while (head < tail) {
            int32_t c = queue[head++];
            int cx = c % ns, cy = (c / ns) % ns, cz = c / (ns * ns);
            int nb[6][3] = {{cx + 1, cy, cz}, {cx - 1, cy, cz}, {cx, cy + 1, cz},
                            {cx, cy - 1, cz}, {cx, cy, cz + 1}, {cx, cy, cz - 1}};
            for (int q = 0; q < 6; ++q) {
                int x = (nb[q][0] + ns) % ns, y = (nb[q][1] + ns) % ns, z = (nb[q][2] + ns) % ns;
                int32_t d = x + ns * (y + ns * z);
                if (gas[d] && label[d] < 0) {
                    label[d] = (int32_t)c0;
                    queue[tail++] = d;
                }
            }
        }
        nclusters += 1;
    }
    free(queue);
    return nclusters;
}

/* ------------------------------------------- Nose-Hoover NVT (Sec. 4.1) */

/* Thermostat half step of the reversible (RESPA / Trotter) splitting of the
 * Nose-Hoover equations (thermostat variable zeta with mass Q, position eta):
 *   zeta += dt/4 G, eta += dt/2 zeta, v *= exp(-dt/2 zeta), zeta += dt/4 G',
 * with G = (2 KE - g T) / Q, g = 3 (N - 1) degrees of freedom. */
static void nh_half(int64_t n, double* v, double dt, double temp, double q, double* zeta, double* eta) {
    double ke = 0.0;
    for (int64_t k = 0; k < 3 * n; ++k) ke += v[k] * v[k];
    ke *= 0.5;
    double g = 3.0 * (double)(n - 1);
    *zeta += 0.25 * dt * (2.0 * ke - g * temp) / q;
    *eta += 0.5 * dt * (*zeta);
    double sc = exp(-0.5 * dt * (*zeta));
    for (int64_t k = 0; k < 3 * n; ++k) v[k] = v[k] * sc;
    ke = ke * sc * sc;
    *zeta += 0.25 * dt * (2.0 * ke - g * temp) / q;
}

/* NVT run: each step is a thermostat half step, one velocity-Verlet step (with the
 * list check and rebuild of orc_run) and a thermostat half step. zeta_eta[2] is
 * read and updated. trace (optional) gets the conserved quantity
 * KE + PE + Q zeta^2 / 2 + g T eta at step 0 and every trace_every steps. */
ORC_API int orc_run_nvt(int64_t n, double box, double rc, double skin, double* x, double* v,
                        int64_t nsteps, double dt, double temp, double q, double* zeta_eta,
                        int64_t* rebuilds, double* trace, int64_t trace_every) {
    double zeta = zeta_eta[0], eta = zeta_eta[1];
    double g = 3.0 * (double)(n - 1);
    int64_t ti = 0, rb_total = 0;
    if (trace) {
        double c2, c0, o[5];
        orc_lj_coeffs(rc, &c2, &c0);
        int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
        int64_t cap = n * 128 + 64;
        int32_t* partners = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        orc_wrap(n, box, x);
        orc_build_list(n, box, rc + skin, x, start, partners, cap);
        orc_observables_list(n, box, rc, c2, c0, x, v, start, partners, o);
        trace[ti++] = o[0] + o[2] + 0.5 * q * zeta * zeta + g * temp * eta;
        free(start);
        free(partners);
    }
    for (int64_t step = 1; step <= nsteps; ++step) {
        nh_half(n, v, dt, temp, q, &zeta, &eta);
        int64_t rb = 0;
        int r = orc_run(n, box, rc, skin, x, v, 1, dt, &rb, NULL, 0);
        if (r) return r;
        rb_total += rb;
        nh_half(n, v, dt, temp, q, &zeta, &eta);
        if (trace && trace_every > 0 && step % trace_every == 0) {
            double c2, c0, o[5];
            orc_lj_coeffs(rc, &c2, &c0);
            int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
            int64_t cap = n * 128 + 64;
            int32_t* partners = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
            orc_build_list(n, box, rc + skin, x, start, partners, cap);
            orc_observables_list(n, box, rc, c2, c0, x, v, start, partners, o);
            trace[ti++] = o[0] + o[2] + 0.5 * q * zeta * zeta + g * temp * eta;
            free(start);
            free(partners);
        }
    }
    zeta_eta[0] = zeta;
    zeta_eta[1] = eta;
    if (rebuilds) *rebuilds = rb_total;
    return 0;
}
