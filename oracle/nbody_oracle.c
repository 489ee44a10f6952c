/*
 * nbody_oracle.c -- CPU oracle for NBSymple's direct-summation method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load, call or
 * link this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library; the two meet only through the seeded initial conditions.
 *
 * Plain, slow, obviously correct: double precision, loops in the order the
 * paper writes its sums, no blocking, no reordering.  Built with
 * -ffp-contract=off and without -ffast-math so every operation rounds once,
 * as written.  OpenMP parallelises only over independent particles i; each
 * per-i sum keeps its serial j order, so results do not depend on the thread
 * count.
 *
 * Conventions (readings of the paper, listed with the design notes):
 *   - accelerations, not forces: the mass m_i of eq. 2 / eq. 5 is divided
 *     out, and eq. 3 adds the external term as an acceleration;
 *   - attractive gravity with potential Phi = -U (U of eq. 4 is positive);
 *   - the j = i term is always skipped (eq. 2); for eps > 0 it is exactly
 *     zero anyway (remark after eq. 5);
 *   - the external field is a Miyamoto-Nagai disk plus a Plummer bulge,
 *     axisymmetric like the disk of the paper's galactic model (Sect. 3),
 *     plus an optional point mass at the galactic centre, Plummer-softened
 *     by eps_bh: the massive black hole of the collision runs of Sect. 6.2,
 *     read as a static central mass.
 *
 * Every function is pinned to something other than itself (the CPU tests of
 * the oracle; the same pins are run against planted mistakes, each of which
 * must fail one); none is "parity unpinned":
 *   orc_accel_int     two-body and n-gon ring closed forms, shells, zero net
 *                     force and torque, translation / rotation / scaling,
 *                     -grad W by differences, Plummer mean field, 60-digit
 *                     brute force within a rounding bound;
 *   orc_accel_int_at  equals orc_accel_int bit for bit on the bodies asked;
 *   orc_ext_phi, orc_ext_accel(_one)  -grad Phi by differences, limits,
 *                     symmetries, scaling laws, v_c closed form, 60-digit
 *                     closed form, black hole = Plummer sphere of its scale;
 *   orc_accel         pair sum plus field (eq. 3), lone body feels the field;
 *   orc_energy        two-body closed forms, -grad W and -grad W_ext, virial
 *                     ratios, 60-digit W;
 *   orc_torque        closed form, dL/dt = M_ext along a step;
 *   orc_run           Kepler orbits at orders 2 and 6 against Kepler's
 *                     equation, energy error scaling, time reversal,
 *                     conservation laws, straight-line free motion.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double G;       /* gravitational constant */
    double eps;     /* softening length, eq. 4-5 (0 = unsoftened eq. 2) */
    int ext_on;     /* 1: add the external field of eq. 3 */
    double Md, ad, bd;  /* Miyamoto-Nagai disk mass, scale length, scale height */
    double Mb, ab;      /* Plummer bulge mass and scale */
    double Mbh, eps_bh; /* central point mass and its softening (0: none) */
} orc_params;

int orc_abi_version(void) { return 1; }

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Internal acceleration, eq. 2 (eps = 0) and eq. 5 (eps > 0), divided by m_i:
 *   a_i = G sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}.
 * pos is (n,3) row-major, acc is written (n,3).
 */
void orc_accel_int(int64_t n, const double *pos, const double *mass,
                   double G, double eps, double *acc)
{
    const double eps2 = eps * eps;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double ax = 0.0, ay = 0.0, az = 0.0;
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = pos[3 * j] - xi;
            const double dy = pos[3 * j + 1] - yi;
            const double dz = pos[3 * j + 2] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            const double r = sqrt(r2);
            const double w = mass[j] / (r2 * r);
            ax += w * dx;
            ay += w * dy;
            az += w * dz;
        }
        acc[3 * i] = G * ax;
        acc[3 * i + 1] = G * ay;
        acc[3 * i + 2] = G * az;
    }
}

/*
 * The same sum as orc_accel_int (eq. 5 / eq. 2), evaluated only for the k
 * bodies listed in idx: acc receives k rows.  Lets full-size outputs be
 * checked on a sample of bodies.
 */
void orc_accel_int_at(int64_t n, const double *pos, const double *mass, double G,
                      double eps, int64_t k, const int64_t *idx, double *acc)
{
    const double eps2 = eps * eps;
    int64_t q;
#pragma omp parallel for schedule(static)
    for (q = 0; q < k; ++q) {
        const int64_t i = idx[q];
        double ax = 0.0, ay = 0.0, az = 0.0;
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = pos[3 * j] - xi;
            const double dy = pos[3 * j + 1] - yi;
            const double dz = pos[3 * j + 2] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            const double r = sqrt(r2);
            const double w = mass[j] / (r2 * r);
            ax += w * dx;
            ay += w * dy;
            az += w * dz;
        }
        acc[3 * q] = G * ax;
        acc[3 * q + 1] = G * ay;
        acc[3 * q + 2] = G * az;
    }
}

/*
 * External potential Phi(x) (per unit mass), the smooth galactic term of
 * eq. 3 with F_ext = -grad Phi:
 *   Phi = -G Md / sqrt(R^2 + (ad + sqrt(z^2 + bd^2))^2) - G Mb / sqrt(r^2 + ab^2)
 *         - G Mbh / sqrt(r^2 + eps_bh^2).
 */
double orc_ext_phi(const orc_params *p, const double *x)
{
    const double R2 = x[0] * x[0] + x[1] * x[1];
    const double s = sqrt(x[2] * x[2] + p->bd * p->bd);
    const double D = sqrt(R2 + (p->ad + s) * (p->ad + s));
    const double rb = sqrt(R2 + x[2] * x[2] + p->ab * p->ab);
    const double rh = sqrt(R2 + x[2] * x[2] + p->eps_bh * p->eps_bh);
    const double ph = p->Mbh > 0 ? p->G * p->Mbh / rh : 0.0;   /* no black hole: no term */
    return -p->G * p->Md / D - p->G * p->Mb / rb - ph;
}

/* External acceleration a = -grad Phi of the potential above, in closed form. */
void orc_ext_accel_one(const orc_params *p, const double *x, double *a)
{
    const double R2 = x[0] * x[0] + x[1] * x[1];
    const double s = sqrt(x[2] * x[2] + p->bd * p->bd);
    const double D2 = R2 + (p->ad + s) * (p->ad + s);
    const double D3 = D2 * sqrt(D2);
    const double rb2 = R2 + x[2] * x[2] + p->ab * p->ab;
    const double rb3 = rb2 * sqrt(rb2);
    const double rh2 = R2 + x[2] * x[2] + p->eps_bh * p->eps_bh;
    const double rh3 = rh2 * sqrt(rh2);
    const double kd = p->G * p->Md / D3;
    const double kb = p->G * p->Mb / rb3;
    const double kh = p->Mbh > 0 ? p->G * p->Mbh / rh3 : 0.0;
    a[0] = -kd * x[0] - kb * x[0] - kh * x[0];
    a[1] = -kd * x[1] - kb * x[1] - kh * x[1];
    a[2] = -kd * x[2] * (p->ad + s) / s - kb * x[2] - kh * x[2];
}

void orc_ext_accel(int64_t n, const double *pos, const orc_params *p, double *acc)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) orc_ext_accel_one(p, pos + 3 * i, acc + 3 * i);
}

/* Total acceleration of eq. 3: internal sum plus (if enabled) external field. */
void orc_accel(int64_t n, const double *pos, const double *mass,
               const orc_params *p, double *acc)
{
    orc_accel_int(n, pos, mass, p->G, p->eps, acc);
    if (p->ext_on) {
        int64_t i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < n; ++i) {
            double ae[3];
            orc_ext_accel_one(p, pos + 3 * i, ae);
            acc[3 * i] += ae[0];
            acc[3 * i + 1] += ae[1];
            acc[3 * i + 2] += ae[2];
        }
    }
}

/*
 * Diagnostics of Sect. 5.1 (eq. 9-10 use E and L):
 *   out[0] K     = 1/2 sum m_i |v_i|^2
 *   out[1] W     = -G sum_{i<j} m_i m_j / sqrt(|r_ij|^2 + eps^2)   (eq. 4)
 *   out[2] W_ext = sum m_i Phi(r_i)  (0 when the field is off)
 *   out[3] E     = K + W + W_ext
 *   out[4..6] P  = sum m_i v_i
 *   out[7..9] L  = sum m_i r_i x v_i
 * Pair partial sums are stored per i and added serially in i order.
 */
void orc_energy(int64_t n, const double *pos, const double *vel,
                const double *mass, const orc_params *p, double *out)
{
    const double eps2 = p->eps * p->eps;
    double *wi = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int64_t i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            const double dx = pos[3 * j] - pos[3 * i];
            const double dy = pos[3 * j + 1] - pos[3 * i + 1];
            const double dz = pos[3 * j + 2] - pos[3 * i + 2];
            s += mass[j] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
        }
        wi[i] = mass[i] * s;
    }
    double K = 0.0, W = 0.0, Wext = 0.0;
    double P[3] = {0.0, 0.0, 0.0}, L[3] = {0.0, 0.0, 0.0};
    for (i = 0; i < n; ++i) {
        const double *x = pos + 3 * i, *v = vel + 3 * i;
        const double m = mass[i];
        K += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        W += wi[i];
        if (p->ext_on) Wext += m * orc_ext_phi(p, x);
        P[0] += m * v[0];
        P[1] += m * v[1];
        P[2] += m * v[2];
        L[0] += m * (x[1] * v[2] - x[2] * v[1]);
        L[1] += m * (x[2] * v[0] - x[0] * v[2]);
        L[2] += m * (x[0] * v[1] - x[1] * v[0]);
    }
    free(wi);
    W = -p->G * W;
    out[0] = K;
    out[1] = W;
    out[2] = Wext;
    out[3] = K + W + Wext;
    out[4] = P[0]; out[5] = P[1]; out[6] = P[2];
    out[7] = L[0]; out[8] = L[1]; out[9] = L[2];
}

/* External torque, eq. 8, with F_ext read as m_i times the field acceleration:
 *   M_ext = sum m_i r_i x a_ext(r_i). */
void orc_torque(int64_t n, const double *pos, const double *mass,
                const orc_params *p, double *out)
{
    double M[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        double a[3];
        const double *x = pos + 3 * i;
        orc_ext_accel_one(p, x, a);
        M[0] += mass[i] * (x[1] * a[2] - x[2] * a[1]);
        M[1] += mass[i] * (x[2] * a[0] - x[0] * a[2]);
        M[2] += mass[i] * (x[0] * a[1] - x[1] * a[0]);
    }
    out[0] = M[0]; out[1] = M[1]; out[2] = M[2];
}

/* ---- Time integration (Sect. 3.1) ------------------------------------- */

static void drift(int64_t n, double *pos, const double *vel, double h)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < 3 * n; ++k) pos[k] += h * vel[k];
}

static void kick(int64_t n, double *vel, const double *acc, double h)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < 3 * n; ++k) vel[k] += h * acc[k];
}

/*
 * Second-order leapfrog, drift-kick-drift form, one step of length h:
 *   r += (h/2) v;  v += h a(r);  r += (h/2) v.
 * acc is caller scratch of size 3n.
 */
static void leapfrog(int64_t n, double *pos, double *vel, const double *mass,
                     const orc_params *p, double h, double *acc)
{
    drift(n, pos, vel, 0.5 * h);
    orc_accel(n, pos, mass, p, acc);
    kick(n, vel, acc, h);
    drift(n, pos, vel, 0.5 * h);
}

/*
 * Sixth-order symplectic step (SI6A of Kinoshita, Yoshida & Nakai 1991, first
 * column of their Table 1, i.e. Yoshida's 1990 "solution A"): the symmetric
 * product of seven leapfrog steps with weights w3 w2 w1 w0 w1 w2 w3, where
 * w0 = 1 - 2 (w1 + w2 + w3).  Seven force evaluations per step (Sect. 3.1).
 * Written as seven literal leapfrog steps; adjacent half drifts are not merged.
 */
static const double SI6A_W1 = -1.17767998417887;
static const double SI6A_W2 = 0.235573213359357;
static const double SI6A_W3 = 0.784513610477560;

void orc_si6a_weights(double *w)
{
    w[1] = SI6A_W1;
    w[2] = SI6A_W2;
    w[3] = SI6A_W3;
    w[0] = 1.0 - 2.0 * (SI6A_W1 + SI6A_W2 + SI6A_W3);
}

static void sixth_order(int64_t n, double *pos, double *vel, const double *mass,
                        const orc_params *p, double h, double *acc)
{
    double w[4];
    orc_si6a_weights(w);
    const int seq[7] = {3, 2, 1, 0, 1, 2, 3};
    for (int k = 0; k < 7; ++k) leapfrog(n, pos, vel, mass, p, w[seq[k]] * h, acc);
}

/*
 * Advance (pos, vel) in place by nsteps steps of length h with the scheme of
 * the given order (2 or 6).  Returns 0, or -1 on a bad argument.
 */
int orc_run(int64_t n, double *pos, double *vel, const double *mass,
            const orc_params *p, int order, double h, int64_t nsteps)
{
    if (order != 2 && order != 6) return -1;
    if (n < 0 || nsteps < 0) return -1;
    double *acc = (double *)malloc((size_t)(n > 0 ? 3 * n : 1) * sizeof(double));
    if (!acc) return -1;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (order == 2)
            leapfrog(n, pos, vel, mass, p, h, acc);
        else
            sixth_order(n, pos, vel, mass, p, h, acc);
    }
    free(acc);
    return 0;
}
