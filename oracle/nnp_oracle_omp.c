/*
 * nnp_oracle_omp.c -- the oracle's full energy and forces with its per-atom
 * loops spread over OpenMP threads, for the benchmark's timed CPU baseline.
 *
 * TEST INFRASTRUCTURE ONLY, like nnp_oracle.c, which this file includes
 * whole: every atom's descriptor, network and force terms come from the
 * oracle's own functions, evaluated as there.  What differs from
 * or_energy_forces is the grouping of two sums: the energy is summed per
 * thread and then across threads, and each thread adds its atoms' force
 * terms into its own array before the arrays are added up.  Results agree
 * with the single-threaded oracle to rounding (tests/test_oracle_omp.py).
 * The pair list and its per-atom lists are built single-threaded, as there.
 */
#define OR_TLS _Thread_local
#include "nnp_oracle.c"

#include <omp.h>

int or_omp_threads(void) { return omp_get_max_threads(); }

/* As or_energy_forces (orthorhombic box or NULL), without G. */
int or_energy_forces_omp(const oracle_model *m, int n, const double *pos, const int *species,
                         const double *box, double *E, double *Ei, double *F) {
    const int D = or_aev_length(m);
    const double rmax = m->rc_r > m->rc_a ? m->rc_r : m->rc_a;
    int *pi, *pj;
    double *pd;
    long np = build_pairs(n, pos, box, rmax, &pi, &pj, &pd);
    nbr_csr rad, ang;
    csr_build(&rad, n, np, pi, pj, pd, m->rc_r);
    csr_build(&ang, n, np, pi, pj, pd, m->rc_a);
    double *G = (double *)malloc(sizeof(double) * (size_t)n * D + 8);
    double *dG = (double *)malloc(sizeof(double) * (size_t)n * D + 8);
    double Etot = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : Etot)
    for (int i = 0; i < n; ++i) {
        aev_atom(m, species, &rad, &ang, i, G + (size_t)i * D);
        const double e = or_mlp(m, species[i], G + (size_t)i * D, dG + (size_t)i * D);
        if (Ei) Ei[i] = e;
        Etot += e;
    }
    *E = Etot;
    const int nt = omp_get_max_threads();
    const size_t stride = (size_t)n * 3 + 3;
    double *acc = (double *)calloc(stride * (size_t)nt, sizeof(double));
#pragma omp parallel
    {
        double *mine = acc + stride * (size_t)omp_get_thread_num();
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) scatter_atom(m, species, &rad, &ang, i, dG + (size_t)i * D, mine);
    }
#pragma omp parallel for schedule(static)
    for (long q = 0; q < 3L * n; ++q) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += acc[stride * (size_t)t + q];
        F[q] = -s;
    }
    free(acc); free(G); free(dG);
    csr_free(&rad); csr_free(&ang);
    free(pi); free(pj); free(pd);
    return 0;
}
