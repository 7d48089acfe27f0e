/*
 * titan_oracle_omp.c -- the FP64 oracle's time step spread over all host cores.
 *
 * TEST INFRASTRUCTURE ONLY, like titan_oracle.c: the benchmark's CPU-baseline
 * leg and the tests load it; the product library never links, loads or calls
 * it, and it shares nothing with the CUDA path.
 *
 * It computes the same step as titan_oracle.c (Sec. III-B, Eq. 1; the planes,
 * friction and constraints of Sec. III-A) and reuses that file's definitions
 * (included below), but organises the spring pass per mass: mass i walks the
 * springs that end on it, in ascending spring index, evaluates each one from
 * the spring's own orientation (d = x_j - x_i, exactly as the serial pass
 * does) and adds +f u when it is the spring's first end, -f u when it is the
 * second.  The serial pass adds to mass i the same products in the same
 * ascending spring order, so the two give bit-identical forces and
 * trajectories (with -ffp-contract=off); no two threads write the same mass,
 * so no atomics are needed.  The mass pass is the serial one, applied to
 * contiguous ranges of masses.
 */
#include "titan_oracle.c"

#include <omp.h>

/* Per-mass incidence of the springs: rowptr [n + 1]; entry r of row i is
 * (s << 1) | end, end = 0 if mass i is ends[2 s], 1 if it is ends[2 s + 1];
 * rows list springs in ascending s.  ent holds 2 s entries. */
void titan_oracle_incidence(const oracle_system *sys, int64_t *rowptr, uint64_t *ent)
{
    const int64_t n = sys->n_masses, S = sys->n_springs;
    for (int64_t i = 0; i <= n; ++i) rowptr[i] = 0;
    for (int64_t s = 0; s < S; ++s) {
        ++rowptr[sys->ends[2 * s] + 1];
        ++rowptr[sys->ends[2 * s + 1] + 1];
    }
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) cur[i] = rowptr[i];
    for (int64_t s = 0; s < S; ++s) {         /* ascending s: rows come out sorted */
        ent[cur[sys->ends[2 * s]]++] = ((uint64_t)s << 1) | 0u;
        ent[cur[sys->ends[2 * s + 1]]++] = ((uint64_t)s << 1) | 1u;
    }
    free(cur);
}

/* Force on one mass from every spring in its row (the serial spring pass's
 * arithmetic, gathered). */
static void gather_force(const oracle_system *sys, const double *x, const double *v, double t,
                         const int64_t *rowptr, const uint64_t *ent, int64_t m, double *Fm)
{
    Fm[0] = Fm[1] = Fm[2] = 0.0;
    for (int64_t r = rowptr[m]; r < rowptr[m + 1]; ++r) {
        const int64_t s = (int64_t)(ent[r] >> 1);
        const int second = (int)(ent[r] & 1u);
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
        if (second) {
            for (int a = 0; a < 3; ++a) Fm[a] -= f * u[a];
        } else {
            for (int a = 0; a < 3; ++a) Fm[a] += f * u[a];
        }
    }
}

/* n_steps time steps on `threads` threads (0: the OpenMP default, all
 * cores).  F is [n][3] scratch; rowptr/ent from titan_oracle_incidence.
 * Returns the number of threads used. */
int titan_oracle_run_parallel(const oracle_system *sys, double *x, double *v, int64_t step0, int64_t n_steps,
                              double *F, const int64_t *rowptr, const uint64_t *ent, int threads)
{
    const int64_t n = sys->n_masses;
    int used = 1;
#pragma omp parallel num_threads(threads > 0 ? threads : omp_get_max_threads())
    {
#pragma omp single
        used = omp_get_num_threads();
        const int nt = omp_get_num_threads(), me = omp_get_thread_num();
        const int64_t i0 = n * me / nt, i1 = n * (me + 1) / nt;
        oracle_system part = *sys;             /* the serial mass pass on [i0, i1) */
        part.n_masses = i1 - i0;
        part.mass = sys->mass + i0;
        part.fixed = sys->fixed ? sys->fixed + i0 : NULL;
        for (int64_t k = 0; k < n_steps; ++k) {
            const double t = (double)(step0 + k) * sys->dt;
            for (int64_t m = i0; m < i1; ++m) gather_force(sys, x, v, t, rowptr, ent, m, F + 3 * m);
#pragma omp barrier
            titan_oracle_mass_update(&part, x + 3 * i0, v + 3 * i0, F + 3 * i0);
#pragma omp barrier
        }
    }
    return used;
}

int titan_oracle_max_threads(void) { return omp_get_max_threads(); }
