/*
 * titan_oracle.c -- plain, slow FP64 CPU simulator of one spring-mass time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the correctness oracle for the CUDA path.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load or call it.  The product library never links, loads or calls it, and
 * the two share no code, header, table or helper.
 *
 * What it computes (Austin et al., "Titan", Sec. III-B, Eq. 1): a time step is
 * one pass over every spring, each applying its Hooke force to both of its end
 * masses, followed by one pass over every mass, each integrated under the sum of
 * the forces it received (Sec. III-A: masses are also subject to gravity, to
 * solid planes with friction, and to constraints).
 *
 * Readings of points the paper leaves open:
 *  - Spring law.  Eq. 1 prints F = k(x1 - x2); read as Hooke's law on the
 *    extension along the spring axis, f = k(l - L), with L the rest length,
 *    plus an axial dashpot c * ((v_j - v_i) . u).  u is the unit vector from
 *    mass i to mass j; mass i receives +f u and mass j receives -f u.
 *  - A spring of zero length (l == 0) has no axis and applies no force.
 *  - Integrator.  Eq. 1 prints dx = xdot dt + xddot dt^2; read as the
 *    velocity-first (symplectic) Euler step v' = v + a dt, x' = x + v' dt,
 *    which is exactly x' = x + v dt + a dt^2.  Forces use (x, v) at the start
 *    of the step.
 *  - Gravity is a constant acceleration g (z is up in every workload here).
 *  - Ground plane z = 0 (Sec. III-A "planes ... frictional forces"): a penalty
 *    normal force k_g * (-z) on a mass below the plane, and Coulomb friction
 *    opposing the tangential velocity (v_x, v_y) with magnitude
 *    min(mu * F_n, m |v_t| / dt), so friction alone never reverses v_t in a
 *    step.  Both use the state at the start of the step.
 *  - Fixed masses (Sec. III-A/C constraints) keep their position, have zero
 *    velocity and ignore every force.
 *  - Actuation mode 1: L(t) = L0 (1 + A sin(2 pi f t + phi)).
 *    Actuation mode 2 (Sec. IV-B, Eqs. 3-5, the worm): L(t) = L0 (1 + c
 *    sin(omega tau)), tau = (t - t_o) mod t_p taken as the floor modulo,
 *    tau in [0, t_p).  Per spring, act_a holds A (or c) and act_b holds phi
 *    (or t_o).
 *  - Time at step n is t_n = n * dt (the step's start).
 *
 * Every sum is taken in input order: forces by spring index, masses by index.
 * Built with -ffp-contract=off so that x86 and Arm hosts round identically.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

/* The layout of this struct is mirrored by the ctypes wrapper in this folder. */
typedef struct {
    int64_t n_masses;
    int64_t n_springs;
    const double *mass;      /* [n]                                   */
    const uint8_t *fixed;    /* [n] or NULL (no fixed masses)          */
    const uint32_t *ends;    /* [s][2] mass indices i, j               */
    const double *k;         /* [s] stiffness (N/m)                    */
    const double *rest;      /* [s] rest length L0 (m)                 */
    const double *damping;   /* [s] axial dashpot c (N s/m)            */
    const double *act_a;     /* [s] amplitude A (mode 1) / c (mode 2)  */
    const double *act_b;     /* [s] phase phi (mode 1) / t_o (mode 2)  */
    int32_t act_mode;        /* 0 none, 1 sinusoid, 2 worm             */
    int32_t ground;          /* nonzero: ground plane z = 0            */
    double act_freq;         /* mode 1: f (Hz)                         */
    double worm_omega;       /* mode 2: omega (rad/s)                  */
    double worm_period;      /* mode 2: t_p (s)                        */
    double dt;               /* time step (s)                          */
    double gravity[3];       /* m/s^2                                  */
    double ground_k;         /* penalty stiffness k_g (N/m)            */
    double mu;               /* Coulomb coefficient                    */
} oracle_system;

static const double kPi = 3.14159265358979323846;

/* Rest length of spring s at time t: Sec. IV-B Eqs. 3-4 (worm) or the
 * sinusoidal form L0 (1 + A sin(2 pi f t + phi)). */
double titan_oracle_rest_length(const oracle_system *sys, int64_t s, double t)
{
    double L0 = sys->rest[s];
    if (sys->act_mode == 1 && sys->act_a) {
        return L0 * (1.0 + sys->act_a[s] * sin(2.0 * kPi * sys->act_freq * t + sys->act_b[s]));
    }
    if (sys->act_mode == 2 && sys->act_a) {
        double tau = t - sys->act_b[s];                            /* Eq. 3: T - t_o   */
        tau = tau - sys->worm_period * floor(tau / sys->worm_period); /* mod t_p         */
        return L0 * (1.0 + sys->act_a[s] * sin(sys->worm_omega * tau)); /* Eq. 4        */
    }
    return L0;
}

/* The spring pass of Sec. III-B: F[i] gets the sum of the forces of every
 * spring that ends on mass i.  F is [n][3] and is overwritten. */
void titan_oracle_spring_forces(const oracle_system *sys, const double *x, const double *v,
                                int64_t step, double *F)
{
    const double t = (double)step * sys->dt;
    memset(F, 0, sizeof(double) * 3 * (size_t)sys->n_masses);
    for (int64_t s = 0; s < sys->n_springs; ++s) {
        const int64_t i = sys->ends[2 * s + 0];
        const int64_t j = sys->ends[2 * s + 1];
        const double L = titan_oracle_rest_length(sys, s, t);
        double d[3], dv[3];
        for (int a = 0; a < 3; ++a) {
            d[a] = x[3 * j + a] - x[3 * i + a];
            dv[a] = v[3 * j + a] - v[3 * i + a];
        }
        const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (len == 0.0) continue;
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = d[a] / len;
        const double rate = dv[0] * u[0] + dv[1] * u[1] + dv[2] * u[2];
        const double f = sys->k[s] * (len - L) + sys->damping[s] * rate;
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += f * u[a];
            F[3 * j + a] -= f * u[a];
        }
    }
}

/* The mass pass of Sec. III-B with the constraints and solids of Sec. III-A:
 * integrate every mass under the spring force it received (F), gravity, and
 * ground contact with friction; fixed masses do not move. */
void titan_oracle_mass_update(const oracle_system *sys, double *x, double *v, const double *F)
{
    const double dt = sys->dt;
    for (int64_t i = 0; i < sys->n_masses; ++i) {
        double *xi = x + 3 * i, *vi = v + 3 * i;
        if (sys->fixed && sys->fixed[i]) {
            vi[0] = vi[1] = vi[2] = 0.0;
            continue;
        }
        const double m = sys->mass[i];
        double a[3];
        for (int c = 0; c < 3; ++c) a[c] = F[3 * i + c] / m + sys->gravity[c];
        if (sys->ground && xi[2] < 0.0) {
            const double Fn = sys->ground_k * (-xi[2]);
            a[2] += Fn / m;
            const double vt = sqrt(vi[0] * vi[0] + vi[1] * vi[1]);
            if (vt > 0.0) {
                double fr = sys->mu * Fn;
                const double cap = m * vt / dt;
                if (cap < fr) fr = cap;
                a[0] -= fr / m * (vi[0] / vt);
                a[1] -= fr / m * (vi[1] / vt);
            }
        }
        for (int c = 0; c < 3; ++c) {
            vi[c] = vi[c] + a[c] * dt;
            xi[c] = xi[c] + vi[c] * dt;
        }
    }
}

/* n_steps full time steps starting at step index step0; x and v are updated
 * in place.  F is caller-provided scratch of [n][3]. */
void titan_oracle_run(const oracle_system *sys, double *x, double *v, int64_t step0,
                      int64_t n_steps, double *F)
{
    for (int64_t n = 0; n < n_steps; ++n) {
        titan_oracle_spring_forces(sys, x, v, step0 + n, F);
        titan_oracle_mass_update(sys, x, v, F);
    }
}

/* ------------------------------------------------------------------ adjoint
 * Reverse-mode derivative of one rollout, used to pin the GPU adjoint.
 * Objective J = sum_i seed_x[i] . x_T[i] + seed_v[i] . v_T[i] after n_steps
 * steps from (x0, v0) at step index step0.  Outputs dJ/dA_s and dJ/dphi_s for
 * the sinusoidal actuation (mode 1) of every spring.  The reverse sweep walks
 * the time steps backwards; within a step it undoes the mass pass (mass by
 * mass) and then the spring pass (spring by spring, in reverse input order).
 * At the kinks (contact on/off, capped/uncapped friction, l = 0) it uses the
 * branch the forward step took.  Every forward state is kept (no
 * checkpointing: the oracle is for small systems).  Returns 0, or -1 if
 * actuation is not mode 1 or memory runs out. */
#include <stdlib.h>

static void adjoint_mass_pass(const oracle_system *sys, const double *x, const double *v,
                              const double *xb_out, const double *vb_out,
                              double *xb, double *vb, double *Fb)
{
    const double dt = sys->dt;
    for (int64_t i = 0; i < sys->n_masses; ++i) {
        const double *xi = x + 3 * i, *vi = v + 3 * i;
        double *xbi = xb + 3 * i, *vbi = vb + 3 * i, *Fbi = Fb + 3 * i;
        if (sys->fixed && sys->fixed[i]) {
            /* x' = x, v' = 0: only the position adjoint passes through */
            for (int c = 0; c < 3; ++c) { xbi[c] = xb_out[3 * i + c]; vbi[c] = 0.0; Fbi[c] = 0.0; }
            continue;
        }
        const double m = sys->mass[i];
        double vtot[3], ab[3];
        for (int c = 0; c < 3; ++c) {
            /* x' = x + v' dt  ->  dJ/dv' gains dt dJ/dx'; v' = v + a dt */
            vtot[c] = vb_out[3 * i + c] + dt * xb_out[3 * i + c];
            xbi[c] = xb_out[3 * i + c];
            vbi[c] = vtot[c];
            ab[c] = dt * vtot[c];
            Fbi[c] = ab[c] / m;          /* a = F / m + g + contact */
        }
        if (sys->ground && xi[2] < 0.0) {
            const double kgm = sys->ground_k / m;      /* a_z += kg (-z) / m */
            xbi[2] += -kgm * ab[2];
            const double vt = sqrt(vi[0] * vi[0] + vi[1] * vi[1]);
            if (vt > 0.0) {
                const double w[2] = {vi[0] / vt, vi[1] / vt};
                /* the forward step's branch: capped iff m vt / dt < mu Fn */
                const double Fn = sys->ground_k * (-xi[2]);
                const int capped = m * vt / dt < sys->mu * Fn;
                const double fr = capped ? vt / dt : sys->mu * Fn / m;     /* |friction| / m */
                /* a_t -= fr w */
                const double frb = -(ab[0] * w[0] + ab[1] * w[1]);
                const double wb[2] = {-fr * ab[0], -fr * ab[1]};
                double vtb = 0.0;
                if (!capped) xbi[2] += -(sys->mu * sys->ground_k / m) * frb;
                else vtb += frb / dt;
                const double wdot = wb[0] * w[0] + wb[1] * w[1];
                for (int c = 0; c < 2; ++c) vbi[c] += (wb[c] - wdot * w[c]) / vt + vtb * w[c];
            }
        }
    }
}

static void adjoint_spring_pass(const oracle_system *sys, const double *x, const double *v, int64_t step,
                                const double *Fb, double *xb, double *vb, double *ga, double *gb)
{
    const double t = (double)step * sys->dt;
    for (int64_t s = sys->n_springs - 1; s >= 0; --s) {
        const int64_t i = sys->ends[2 * s + 0];
        const int64_t j = sys->ends[2 * s + 1];
        double d[3], dv[3];
        for (int a = 0; a < 3; ++a) {
            d[a] = x[3 * j + a] - x[3 * i + a];
            dv[a] = v[3 * j + a] - v[3 * i + a];
        }
        const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (len == 0.0) continue;
        double u[3], g[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = d[a] / len;
            g[a] = Fb[3 * i + a] - Fb[3 * j + a];     /* F_i += f u, F_j -= f u */
        }
        const double L = titan_oracle_rest_length(sys, s, t);
        const double rate = dv[0] * u[0] + dv[1] * u[1] + dv[2] * u[2];
        const double f = sys->k[s] * (len - L) + sys->damping[s] * rate;
        const double fb = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
        double ub[3];
        for (int a = 0; a < 3; ++a) ub[a] = f * g[a];
        const double lenb = sys->k[s] * fb;
        const double Lb = -sys->k[s] * fb;
        const double rateb = sys->damping[s] * fb;
        for (int a = 0; a < 3; ++a) {
            vb[3 * j + a] += rateb * u[a];
            vb[3 * i + a] -= rateb * u[a];
            ub[a] += rateb * dv[a];
        }
        const double udot = ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2];
        for (int a = 0; a < 3; ++a) {
            const double db = (ub[a] - udot * u[a]) / len + lenb * u[a];
            xb[3 * j + a] += db;
            xb[3 * i + a] -= db;
        }
        /* L = L0 (1 + A sin(2 pi f t + phi)) */
        const double th = 2.0 * kPi * sys->act_freq * t + sys->act_b[s];
        ga[s] += Lb * sys->rest[s] * sin(th);
        gb[s] += Lb * sys->rest[s] * sys->act_a[s] * cos(th);
    }
}

int titan_oracle_adjoint(const oracle_system *sys, const double *x0, const double *v0, int64_t step0,
                         int64_t n_steps, const double *seed_x, const double *seed_v,
                         double *grad_a, double *grad_b, double *x_T, double *v_T)
{
    if (sys->act_mode != 1 || !sys->act_a) return -1;
    const size_t n3 = 3 * (size_t)sys->n_masses;
    double *X = (double *)malloc(sizeof(double) * n3 * (size_t)(n_steps + 1));
    double *V = (double *)malloc(sizeof(double) * n3 * (size_t)(n_steps + 1));
    double *F = (double *)malloc(sizeof(double) * n3);
    double *xb = (double *)malloc(sizeof(double) * n3), *vb = (double *)malloc(sizeof(double) * n3);
    double *xb2 = (double *)malloc(sizeof(double) * n3), *vb2 = (double *)malloc(sizeof(double) * n3);
    if (!X || !V || !F || !xb || !vb || !xb2 || !vb2) {
        free(X); free(V); free(F); free(xb); free(vb); free(xb2); free(vb2);
        return -1;
    }
    memcpy(X, x0, sizeof(double) * n3);
    memcpy(V, v0, sizeof(double) * n3);
    for (int64_t n = 0; n < n_steps; ++n) {
        memcpy(X + n3 * (n + 1), X + n3 * n, sizeof(double) * n3);
        memcpy(V + n3 * (n + 1), V + n3 * n, sizeof(double) * n3);
        titan_oracle_spring_forces(sys, X + n3 * (n + 1), V + n3 * (n + 1), step0 + n, F);
        titan_oracle_mass_update(sys, X + n3 * (n + 1), V + n3 * (n + 1), F);
    }
    if (x_T) memcpy(x_T, X + n3 * n_steps, sizeof(double) * n3);
    if (v_T) memcpy(v_T, V + n3 * n_steps, sizeof(double) * n3);
    for (size_t k = 0; k < n3; ++k) {
        xb[k] = seed_x ? seed_x[k] : 0.0;
        vb[k] = seed_v ? seed_v[k] : 0.0;
    }
    memset(grad_a, 0, sizeof(double) * (size_t)sys->n_springs);
    memset(grad_b, 0, sizeof(double) * (size_t)sys->n_springs);
    for (int64_t n = n_steps - 1; n >= 0; --n) {
        const double *x = X + n3 * n, *v = V + n3 * n;
        adjoint_mass_pass(sys, x, v, xb, vb, xb2, vb2, F);
        adjoint_spring_pass(sys, x, v, step0 + n, F, xb2, vb2, grad_a, grad_b);
        double *tx = xb; xb = xb2; xb2 = tx;
        double *tv = vb; vb = vb2; vb2 = tv;
    }
    free(X); free(V); free(F); free(xb); free(vb); free(xb2); free(vb2);
    return 0;
}
