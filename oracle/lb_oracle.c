/*
 * lb_oracle.c -- plain FP64 CPU reference for the D3Q19 BGK lattice update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; it exists so the tests, the smoke check and the CPU-baseline
 * leg of the benchmark can compare the CUDA library against an independent,
 * obviously correct implementation.  It shares no table, header or helper with
 * the CUDA sources: the velocity set is built here by enumeration, the
 * population order is this file's own, and every step is written as a plain
 * loop in the order of the method.
 *
 * What it computes (arXiv 2409.16781, Sec. 2 "Lattice Boltzmann Method",
 * Eq. 1-3, and Sec. 3.1 for the fused pull / two-array scheme):
 *
 *   f_i(x + c_i, t + 1) = f_i(x, t) - omega (f_i(x, t) - f_i^eq(x, t)) + S_i   (Eq. 1)
 *   f_i^eq = w_i rho (1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u)                  (Eq. 2-3)
 *
 * Readings of the paper taken here (the paper states its method for D2Q9 and
 * names the 3D extension as future work, Sec. 6):
 *   - velocity set D3Q19: all c in {-1,0,1}^3 with |c|^2 <= 2, weights 1/3
 *     (rest), 1/18 (|c|^2 = 1), 1/36 (|c|^2 = 2); c_s^2 = 1/3;
 *   - Eq. 3 is printed with inconsistent powers of c_s; the standard second
 *     order truncation above is used;
 *   - omega = 1/tau;
 *   - the source S_i of Eq. 1 is Guo forcing (Guo, Zheng & Shi 2002) for a
 *     body force per unit mass g (force density rho g), with the half-force
 *     velocity shift u = (sum_i f_i c_i)/rho + g/2;
 *   - walls (Sec. 3.3, lid-driven cavity: no-slip walls, lid moving at u0)
 *     are cells flagged WALL or LID; a fluid cell whose pull source x - c_i is
 *     such a cell takes the halfway bounce-back value f_opp(i)*(x), plus
 *     6 w_i rho_w (c_i . u_lid) with rho_w = 1 when the source is a LID cell;
 *   - the pull (Sec. 3.1: "scattered read" from f^pre, result in f^post) wraps
 *     periodically at the domain edges; solid cells are never written;
 *   - von Karman street (Sec. 3.3 names it; no boundary conditions given):
 *     the inflow and outflow planes are FARFIELD cells held at the free
 *     stream, the equilibrium of density 1 moving at u_lid (lbo_pull).
 *
 * Array layout used by this file: f[q * N + cell], cell = x + nx*(y + ny*z),
 * q in this file's own velocity order (lbo_velocity_set reports it).
 *
 * Two-relaxation-time collision (not in the paper; an alternative collision
 * for tau near 1/2, Ginzburg's TRT): lbo_step_trt relaxes the part of each
 * population even under c -> -c, f+_i = (f_i + f_opp(i))/2, with omega+ =
 * 1/tau and the odd part f-_i = (f_i - f_opp(i))/2 with omega-; the Guo
 * source splits the same way, its even part scaled by (1 - omega+/2) and its
 * odd part by (1 - omega-/2).  omega- = omega+ is BGK.
 */
#include <stddef.h>
#include <stdint.h>
#include <math.h>

#define LBO_Q 19
#define LBO_FLUID 0
#define LBO_WALL 1
#define LBO_LID 2
#define LBO_FARFIELD 3

static int lbo_c[LBO_Q][3];
static double lbo_w[LBO_Q];
static int lbo_opp[LBO_Q];
static int lbo_ready = 0;

/* Build the D3Q19 set by enumerating {-1,0,1}^3 and keeping |c|^2 <= 2. */
static void lbo_build(void)
{
    if (lbo_ready) return;
    int q = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int n2 = cx * cx + cy * cy + cz * cz;
                if (n2 > 2) continue;
                lbo_c[q][0] = cx;
                lbo_c[q][1] = cy;
                lbo_c[q][2] = cz;
                lbo_w[q] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++q;
            }
    for (int i = 0; i < LBO_Q; ++i)
        for (int j = 0; j < LBO_Q; ++j)
            if (lbo_c[j][0] == -lbo_c[i][0] && lbo_c[j][1] == -lbo_c[i][1] &&
                lbo_c[j][2] == -lbo_c[i][2])
                lbo_opp[i] = j;
    lbo_ready = 1;
}

/* Report the velocity set in this file's order: c[19*3], w[19].  Returns 19. */
int lbo_velocity_set(int *c, double *w)
{
    lbo_build();
    for (int i = 0; i < LBO_Q; ++i) {
        c[3 * i + 0] = lbo_c[i][0];
        c[3 * i + 1] = lbo_c[i][1];
        c[3 * i + 2] = lbo_c[i][2];
        w[i] = lbo_w[i];
    }
    return LBO_Q;
}

/* Eq. 2-3: second-order equilibrium. */
void lbo_equilibrium(double rho, const double *u, double *feq)
{
    lbo_build();
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < LBO_Q; ++i) {
        double cu = lbo_c[i][0] * u[0] + lbo_c[i][1] * u[1] + lbo_c[i][2] * u[2];
        feq[i] = lbo_w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* S_i of Eq. 1 as Guo forcing: (1 - omega/2) w_i [3(c_i - u) + 9 (c_i.u) c_i] . F,
 * with F = rho g the force density. */
void lbo_source(double tau, double rho, const double *u, const double *g, double *S)
{
    lbo_build();
    double F[3] = {rho * g[0], rho * g[1], rho * g[2]};
    double pref = 1.0 - 0.5 / tau;
    for (int i = 0; i < LBO_Q; ++i) {
        double cu = lbo_c[i][0] * u[0] + lbo_c[i][1] * u[1] + lbo_c[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += (3.0 * (lbo_c[i][a] - u[a]) + 9.0 * cu * lbo_c[i][a]) * F[a];
        S[i] = pref * lbo_w[i] * s;
    }
}

static inline size_t lbo_idx(int x, int y, int z, int nx, int ny)
{
    return (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
}

static inline int lbo_wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

/* Streaming (pull) with the boundary rules: the 19 populations arriving at
 * fluid cell (x,y,z) from post-collision array A.
 * FARFIELD cells (the inflow and outflow planes of the von Karman street use
 * case, flow past a cylinder, Sec. 3.3, whose boundary conditions the paper
 * does not give): the free stream -- the value arriving from a far-field
 * source is the equilibrium f^eq_i(rho = 1, U) of Eq. 2-3 with U = u_lid,
 * whatever the fluid sends out (an absorbing, Dirichlet condition on both
 * density and velocity). */
static void lbo_pull(int nx, int ny, int nz, const double *ulid, const uint8_t *flags,
                     const double *A, int x, int y, int z, double *f)
{
    size_t N = (size_t)nx * ny * nz;
    size_t cell = lbo_idx(x, y, z, nx, ny);
    double f_free[LBO_Q];
    if (flags != NULL) lbo_equilibrium(1.0, ulid, f_free);
    for (int i = 0; i < LBO_Q; ++i) {
        int sx = lbo_wrap(x - lbo_c[i][0], nx);
        int sy = lbo_wrap(y - lbo_c[i][1], ny);
        int sz = lbo_wrap(z - lbo_c[i][2], nz);
        size_t src = lbo_idx(sx, sy, sz, nx, ny);
        if (flags != NULL && flags[src] == LBO_FARFIELD) {
            f[i] = f_free[i];
            continue;
        }
        if (flags == NULL || flags[src] == LBO_FLUID) {
            f[i] = A[(size_t)i * N + src];
        } else {
            f[i] = A[(size_t)lbo_opp[i] * N + cell];
            if (flags[src] == LBO_LID) {
                double cu = lbo_c[i][0] * ulid[0] + lbo_c[i][1] * ulid[1] + lbo_c[i][2] * ulid[2];
                f[i] += 6.0 * lbo_w[i] * 1.0 * cu; /* rho_w = 1 */
            }
        }
    }
}

/* Density and (half-force shifted) velocity of a set of populations. */
static void lbo_macro(const double *f, const double *g, double *rho, double *u)
{
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < LBO_Q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * lbo_c[i][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r + 0.5 * g[a];
}

/* A <- f^eq(rho, u) at every cell (rho, u may be NULL: rho = 1, u = 0).
 * u is SoA: u[a*N + cell]. */
void lbo_init(int nx, int ny, int nz, const double *rho, const double *u, double *A)
{
    lbo_build();
    size_t N = (size_t)nx * ny * nz;
    for (size_t cell = 0; cell < N; ++cell) {
        double r = rho ? rho[cell] : 1.0;
        double uc[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int a = 0; a < 3; ++a) uc[a] = u[(size_t)a * N + cell];
        double feq[LBO_Q];
        lbo_equilibrium(r, uc, feq);
        for (int i = 0; i < LBO_Q; ++i) A[(size_t)i * N + cell] = feq[i];
    }
}

/* One fused pull step of Eq. 1: B <- collide(stream(A)) at every fluid cell.
 * Solid cells of B are left as they are. */
void lbo_step(int nx, int ny, int nz, double tau, const double *ulid, const double *g,
              const uint8_t *flags, const double *A, double *B)
{
    lbo_build();
    size_t N = (size_t)nx * ny * nz;
    double omega = 1.0 / tau;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cell = lbo_idx(x, y, z, nx, ny);
                if (flags && flags[cell] != LBO_FLUID) continue;
                double f[LBO_Q], feq[LBO_Q], S[LBO_Q], rho, u[3];
                lbo_pull(nx, ny, nz, ulid, flags, A, x, y, z, f);      /* streaming */
                lbo_macro(f, g, &rho, u);                               /* moments */
                lbo_equilibrium(rho, u, feq);                           /* Eq. 2-3 */
                lbo_source(tau, rho, u, g, S);                          /* S_i */
                for (int i = 0; i < LBO_Q; ++i)                         /* Eq. 1 */
                    B[(size_t)i * N + cell] = f[i] - omega * (f[i] - feq[i]) + S[i];
            }
}

/* Unscaled Guo term G_i = w_i [3(c_i - u) + 9 (c_i.u) c_i] . F, F = rho g. */
static void lbo_guo_unscaled(double rho, const double *u, const double *g, double *G)
{
    double F[3] = {rho * g[0], rho * g[1], rho * g[2]};
    for (int i = 0; i < LBO_Q; ++i) {
        double cu = lbo_c[i][0] * u[0] + lbo_c[i][1] * u[1] + lbo_c[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += (3.0 * (lbo_c[i][a] - u[a]) + 9.0 * cu * lbo_c[i][a]) * F[a];
        G[i] = lbo_w[i] * s;
    }
}

/* One fused pull step with the TRT collision (omega+ = 1/tau, omega-). */
void lbo_step_trt(int nx, int ny, int nz, double tau, double omega_minus, const double *ulid,
                  const double *g, const uint8_t *flags, const double *A, double *B)
{
    lbo_build();
    size_t N = (size_t)nx * ny * nz;
    double wp = 1.0 / tau, wm = omega_minus;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cell = lbo_idx(x, y, z, nx, ny);
                if (flags && flags[cell] != LBO_FLUID) continue;
                double f[LBO_Q], feq[LBO_Q], G[LBO_Q], rho, u[3];
                lbo_pull(nx, ny, nz, ulid, flags, A, x, y, z, f);
                lbo_macro(f, g, &rho, u);
                lbo_equilibrium(rho, u, feq);
                lbo_guo_unscaled(rho, u, g, G);
                for (int i = 0; i < LBO_Q; ++i) {
                    int o = lbo_opp[i];
                    double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
                    double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
                    double gp = 0.5 * (G[i] + G[o]), gm = 0.5 * (G[i] - G[o]);
                    B[(size_t)i * N + cell] = f[i] - wp * (fp - ep) - wm * (fm - em)
                                              + (1.0 - 0.5 * wp) * gp + (1.0 - 0.5 * wm) * gm;
                }
            }
}

/* As lbo_run, with the TRT collision. */
int lbo_run_trt(int nx, int ny, int nz, double tau, double omega_minus, const double *ulid,
                const double *g, const uint8_t *flags, double *A, double *B, int n)
{
    for (int t = 0; t < n; ++t) {
        if (t % 2 == 0)
            lbo_step_trt(nx, ny, nz, tau, omega_minus, ulid, g, flags, A, B);
        else
            lbo_step_trt(nx, ny, nz, tau, omega_minus, ulid, g, flags, B, A);
    }
    return n % 2;
}

/* Run n steps starting from A, alternating A and B; returns the array that
 * holds the result (0: A, 1: B). */
int lbo_run(int nx, int ny, int nz, double tau, const double *ulid, const double *g,
            const uint8_t *flags, double *A, double *B, int n)
{
    for (int t = 0; t < n; ++t) {
        if (t % 2 == 0)
            lbo_step(nx, ny, nz, tau, ulid, g, flags, A, B);
        else
            lbo_step(nx, ny, nz, tau, ulid, g, flags, B, A);
    }
    return n % 2;
}

/* Fields of the lattice whose post-collision array is A: rho and u of the
 * streamed populations at every fluid cell (u SoA, half-force shifted);
 * solid cells get rho = 0, u = 0. */
void lbo_moments(int nx, int ny, int nz, const double *ulid, const double *g,
                 const uint8_t *flags, const double *A, double *rho, double *u)
{
    lbo_build();
    size_t N = (size_t)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cell = lbo_idx(x, y, z, nx, ny);
                double r = 0.0, uc[3] = {0.0, 0.0, 0.0};
                if (!flags || flags[cell] == LBO_FLUID) {
                    double f[LBO_Q];
                    lbo_pull(nx, ny, nz, ulid, flags, A, x, y, z, f);
                    lbo_macro(f, g, &r, uc);
                }
                rho[cell] = r;
                for (int a = 0; a < 3; ++a) u[(size_t)a * N + cell] = uc[a];
            }
}

/* Mass sum(rho) and momentum sum(rho u) over fluid cells. */
void lbo_totals(int nx, int ny, int nz, const double *ulid, const double *g,
                const uint8_t *flags, const double *A, double *out4)
{
    lbo_build();
    double m = 0.0, p[3] = {0.0, 0.0, 0.0};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cell = lbo_idx(x, y, z, nx, ny);
                if (flags && flags[cell] != LBO_FLUID) continue;
                double f[LBO_Q], r, uc[3];
                lbo_pull(nx, ny, nz, ulid, flags, A, x, y, z, f);
                lbo_macro(f, g, &r, uc);
                m += r;
                for (int a = 0; a < 3; ++a) p[a] += r * uc[a];
            }
    out4[0] = m;
    out4[1] = p[0];
    out4[2] = p[1];
    out4[3] = p[2];
}
