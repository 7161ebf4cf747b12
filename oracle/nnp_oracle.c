/*
 * nnp_oracle.c -- plain, slow, single-threaded FP64 reference of the NNP
 * energy/force path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  The CUDA library
 * shares no code, header or constant table with it.
 *
 * What it computes (paper: Theory, Eq. 1 and Eq. 2; the descriptor is the
 * ANI atomic environment vector the paper cites for its ANI-2x runs):
 *
 *   E_ML = sum_i E_i,  E_i = MLP_{s_i}(G_i)                  (per-element nets)
 *   F_i  = -dE_ML/dr_i                                        (Eq. 2)
 *
 *   Radial AEV of atom i, neighbour j of species s_j, shift m:
 *     G_i[s_j*nR + m] += 1/4 exp(-eta_R (r_ij - R_m)^2) fc(r_ij; Rc_R)
 *   Angular AEV, unordered pair {j,k} of neighbours within Rc_A:
 *     theta' = arccos(0.95 cos theta_ijk)
 *     G_i[nR*S + p(s_j,s_k)*nA*nZ + a*nZ + z] +=
 *        2^(1-zeta) (1 + cos(theta' - theta_z))^zeta
 *        * exp(-eta_A ((r_ij + r_ik)/2 - R_a)^2) fc(r_ij; Rc_A) fc(r_ik; Rc_A)
 *   fc(r; Rc) = 1/2 cos(pi r / Rc) + 1/2 for r < Rc, else 0.
 *   p(s1,s2), s1 <= s2: row-major index of the upper triangle.
 *   MLP: h_l = CELU_alpha(h_{l-1} W_l + b_l), l = 1..L-1; E_i = h W_L + b_L.
 *
 *   Pairs: every (j, periodic image) with |r_j + n.L - r_i| < Rc (strict),
 *   j == i allowed only for a non-zero image; brute force over all images
 *   that can lie within Rc, no minimum-image shortcut.
 *
 *   Force matching: L = 1/(3N) sum_i |F_i - Fref_i|^2 and dL/dtheta,
 *   computed as -d/dtheta of the directional derivative of E along
 *   v = dL/dF (forward-over-reverse through the per-atom networks).
 *
 * All arithmetic is double precision.  Every loop follows the definition in
 * the order written above; nothing is blocked, fused or reordered.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_SPECIES 8
#define OR_MAX_SHF 32
#define OR_MAX_LAYERS 8

/* Storage class of the network's scratch rows: empty here (plain statics,
 * single-threaded); the OpenMP build (nnp_oracle_omp.c) makes them
 * thread-local. */
#ifndef OR_TLS
#define OR_TLS
#endif

typedef struct {
    int n_species;
    int n_rad;     /* radial shifts per neighbour species */
    int n_ang_r;   /* angular radial shifts */
    int n_ang_z;   /* angular sectors */
    double rc_r, eta_r, rc_a, eta_a, zeta;
    double shf_r[OR_MAX_SHF], shf_a[OR_MAX_SHF], shf_z[OR_MAX_SHF];
    int n_layers;                       /* weight layers (4 for 128-160-128-96-1) */
    int width[OR_MAX_LAYERS + 1];       /* width[0] = D, width[n_layers] = 1 */
    double celu_alpha;
    /* W[s*OR_MAX_LAYERS + l]: width[l] x width[l+1], row-major; b[...]: width[l+1] */
    const double *W[OR_MAX_SPECIES * OR_MAX_LAYERS];
    const double *b[OR_MAX_SPECIES * OR_MAX_LAYERS];
} oracle_model;

/* ----------------------------------------------------------------------- */
/* descriptor length and index helpers                                      */

int or_aev_length(const oracle_model *m) {
    int S = m->n_species;
    return m->n_rad * S + m->n_ang_r * m->n_ang_z * S * (S + 1) / 2;
}

static int pair_index(int S, int s1, int s2) {
    if (s1 > s2) { int t = s1; s1 = s2; s2 = t; }
    /* rows 0..s1-1 of the upper triangle hold S, S-1, ..., S-s1+1 entries */
    int before = 0;
    for (int r = 0; r < s1; ++r) before += S - r;
    return before + (s2 - s1);
}

int or_pair_index(int S, int s1, int s2) { return pair_index(S, s1, s2); }

static double fc(double r, double rc) {
    if (r >= rc) return 0.0;
    return 0.5 * cos(M_PI * r / rc) + 0.5;
}

static double dfc(double r, double rc) {
    if (r >= rc) return 0.0;
    return -0.5 * (M_PI / rc) * sin(M_PI * r / rc);
}

/* ----------------------------------------------------------------------- */
/* pairs                                                                     */

static void wrap_positions(int n, const double *pos, const double *box, double *out) {
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double x = pos[3 * i + a];
            if (box) {
                x = x - box[a] * floor(x / box[a]);
                if (x >= box[a]) x -= box[a]; /* floor rounding at the top edge */
                if (x < 0.0) x = 0.0;
            }
            out[3 * i + a] = x;
        }
}

static long emit(long cnt, long cap, int *pi, int *pj, double *pd,
                 int i, int j, const double d[3]) {
    if (cnt < cap) {
        pi[cnt] = i; pj[cnt] = j;
        pd[3 * cnt] = d[0]; pd[3 * cnt + 1] = d[1]; pd[3 * cnt + 2] = d[2];
    }
    return cnt + 1;
}

/* General periodic cell (triclinic): rows of cell are the cell vectors a, b,
 * c (right-handed).  Positions are wrapped through fractional coordinates
 * s = r B^-1 into [0, 1); then every image n = (n0, n1, n2) with |n_d| <=
 * ceil(rc / h_d) + 1 is tried, h_d the cell's height across the other two
 * vectors (d = r_j + n0 a + n1 b + n2 c - r_i), which covers every pair of
 * wrapped atoms within rc.  Returns the number of pairs; writes the first
 * `cap`. */
static double det3(const double *B) {
    return B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
           B[2] * (B[3] * B[7] - B[4] * B[6]);
}

static void cross3(const double *u, const double *v, double *w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

long or_pairs_brute_cell(int n, const double *pos, const double *cell, double rc,
                         long cap, int *pi, int *pj, double *pd) {
    const double V = det3(cell);
    /* inverse by cofactors: Binv[c][d] with s_d = sum_c r_c Binv[c][d] */
    double Binv[9];
    {
        const double *a = cell, *b = cell + 3, *c = cell + 6;
        double bc[3], ca[3], ab[3];
        cross3(b, c, bc); cross3(c, a, ca); cross3(a, b, ab);
        for (int k = 0; k < 3; ++k) {
            Binv[3 * k + 0] = bc[k] / V;
            Binv[3 * k + 1] = ca[k] / V;
            Binv[3 * k + 2] = ab[k] / V;
        }
    }
    int nmax[3];
    for (int d = 0; d < 3; ++d) {
        double w[3];
        cross3(cell + 3 * ((d + 1) % 3), cell + 3 * ((d + 2) % 3), w);
        const double h = V / sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        nmax[d] = (int)ceil(rc / h) + 1;
    }
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        double sf[3];
        for (int d = 0; d < 3; ++d) {
            double t = 0.0;
            for (int c = 0; c < 3; ++c) t += pos[3 * i + c] * Binv[3 * c + d];
            t -= floor(t);
            if (t >= 1.0) t -= 1.0;
            sf[d] = t;
        }
        for (int c = 0; c < 3; ++c) x[3 * i + c] = sf[0] * cell[c] + sf[1] * cell[3 + c] + sf[2] * cell[6 + c];
    }
    long cnt = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
                for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                    for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                        if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;
                        double d[3];
                        for (int c = 0; c < 3; ++c)
                            d[c] = x[3 * j + c] - x[3 * i + c] + n0 * cell[c] + n1 * cell[3 + c] + n2 * cell[6 + c];
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 < rc * rc) cnt = emit(cnt, cap, pi, pj, pd, i, j, d);
                    }
    free(x);
    return cnt;
}

/* All (i, j, image) with |d| < rc, d = r_j + n.L - r_i, by brute force over
 * every image n with |n_a L_a| < rc + L_a.  box = NULL: isolated system.
 * Returns the number of pairs; writes the first `cap` of them. */
long or_pairs_brute(int n, const double *pos, const double *box, double rc,
                    long cap, int *pi, int *pj, double *pd) {
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    wrap_positions(n, pos, box, x);
    int nmax[3] = {0, 0, 0};
    if (box)
        for (int a = 0; a < 3; ++a) nmax[a] = (int)floor(rc / box[a]) + 1;
    long cnt = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
                for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                    for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                        if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;
                        double d[3];
                        d[0] = x[3 * j] - x[3 * i] + (box ? n0 * box[0] : 0.0);
                        d[1] = x[3 * j + 1] - x[3 * i + 1] + (box ? n1 * box[1] : 0.0);
                        d[2] = x[3 * j + 2] - x[3 * i + 2] + (box ? n2 * box[2] : 0.0);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 < rc * rc) cnt = emit(cnt, cap, pi, pj, pd, i, j, d);
                    }
    free(x);
    return cnt;
}

/* Same pair set through a cell list: cells of edge >= rc (one cell if the
 * box is shorter than rc), neighbour cells visited as "virtual" cells
 * k_i + m whose image shift is floor((k_i + m) / nc).  Isolated systems use
 * the brute-force enumeration. */
long or_pairs_cells(int n, const double *pos, const double *box, double rc,
                    long cap, int *pi, int *pj, double *pd) {
    if (!box) return or_pairs_brute(n, pos, box, rc, cap, pi, pj, pd);
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    wrap_positions(n, pos, box, x);
    int nc[3], M[3];
    double ell[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(box[a] / rc);
        if (nc[a] < 1) nc[a] = 1;
        ell[a] = box[a] / nc[a];
        M[a] = (int)ceil(rc / ell[a]);
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int *cell = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *head = (int *)malloc(sizeof(int) * (size_t)ncell);
    int *next = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int (*kc)[3] = malloc(sizeof(int[3]) * (size_t)(n > 0 ? n : 1));
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    /* singly linked lists, built back to front so each list is in index order */
    for (int i = n - 1; i >= 0; --i) {
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor(x[3 * i + a] / ell[a]);
            if (k >= nc[a]) k = nc[a] - 1;
            if (k < 0) k = 0;
            kc[i][a] = k;
        }
        long c = ((long)kc[i][0] * nc[1] + kc[i][1]) * nc[2] + kc[i][2];
        cell[i] = (int)c;
        next[i] = head[c];
        head[c] = i;
    }
    long cnt = 0;
    for (int i = 0; i < n; ++i)
        for (int m0 = -M[0]; m0 <= M[0]; ++m0)
            for (int m1 = -M[1]; m1 <= M[1]; ++m1)
                for (int m2 = -M[2]; m2 <= M[2]; ++m2) {
                    int v[3] = {kc[i][0] + m0, kc[i][1] + m1, kc[i][2] + m2};
                    int k[3], sh[3];
                    for (int a = 0; a < 3; ++a) {
                        sh[a] = (int)floor((double)v[a] / nc[a]);
                        k[a] = v[a] - sh[a] * nc[a];
                    }
                    long c = ((long)k[0] * nc[1] + k[1]) * nc[2] + k[2];
                    for (int j = head[c]; j >= 0; j = next[j]) {
                        if (i == j && sh[0] == 0 && sh[1] == 0 && sh[2] == 0) continue;
                        double d[3];
                        for (int a = 0; a < 3; ++a)
                            d[a] = x[3 * j + a] + sh[a] * box[a] - x[3 * i + a];
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 < rc * rc) cnt = emit(cnt, cap, pi, pj, pd, i, j, d);
                    }
                }
    free(x); free(cell); free(head); free(next); free(kc);
    return cnt;
}

/* ----------------------------------------------------------------------- */
/* per-atom neighbour lists (CSR) built from a pair list                    */

typedef struct {
    int n;
    long *start;   /* n+1 */
    int *j;
    double *d;     /* 3 per entry */
} nbr_csr;

static void csr_build(nbr_csr *c, int n, long np, const int *pi, const int *pj,
                      const double *pd, double rc) {
    c->n = n;
    c->start = (long *)calloc((size_t)n + 1, sizeof(long));
    long keep = 0;
    for (long q = 0; q < np; ++q) {
        double r2 = pd[3 * q] * pd[3 * q] + pd[3 * q + 1] * pd[3 * q + 1] +
                    pd[3 * q + 2] * pd[3 * q + 2];
        if (r2 < rc * rc) { c->start[pi[q] + 1]++; keep++; }
    }
    for (int i = 0; i < n; ++i) c->start[i + 1] += c->start[i];
    c->j = (int *)malloc(sizeof(int) * (size_t)(keep > 0 ? keep : 1));
    c->d = (double *)malloc(sizeof(double) * 3 * (size_t)(keep > 0 ? keep : 1));
    long *fill = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) fill[i] = c->start[i];
    for (long q = 0; q < np; ++q) {
        double r2 = pd[3 * q] * pd[3 * q] + pd[3 * q + 1] * pd[3 * q + 1] +
                    pd[3 * q + 2] * pd[3 * q + 2];
        if (r2 < rc * rc) {
            long w = fill[pi[q]]++;
            c->j[w] = pj[q];
            c->d[3 * w] = pd[3 * q]; c->d[3 * w + 1] = pd[3 * q + 1]; c->d[3 * w + 2] = pd[3 * q + 2];
        }
    }
    free(fill);
}

static void csr_free(nbr_csr *c) { free(c->start); free(c->j); free(c->d); }

/* ----------------------------------------------------------------------- */
/* AEV and its derivatives                                                   */

/* One radial term and its r-derivative. */
static void radial_term(const oracle_model *m, int k, double r, double *t, double *dt) {
    double e = exp(-m->eta_r * (r - m->shf_r[k]) * (r - m->shf_r[k]));
    *t = 0.25 * e * fc(r, m->rc_r);
    *dt = 0.25 * e * (-2.0 * m->eta_r * (r - m->shf_r[k]) * fc(r, m->rc_r) + dfc(r, m->rc_r));
}

/* One angular term T(d_u, d_v) for shift a, sector z; optionally its
 * gradients dT/dd_u and dT/dd_v (3-vectors). */
static double angular_term(const oracle_model *m, int a, int z, const double du[3],
                           const double dv[3], double gu[3], double gv[3]) {
    double ru = sqrt(du[0] * du[0] + du[1] * du[1] + du[2] * du[2]);
    double rv = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double c = (du[0] * dv[0] + du[1] * dv[1] + du[2] * dv[2]) / (ru * rv);
    double theta = acos(0.95 * c);
    double base = 1.0 + cos(theta - m->shf_z[z]);
    double A = pow(2.0, 1.0 - m->zeta) * pow(base, m->zeta);
    double rbar = 0.5 * (ru + rv);
    double B = exp(-m->eta_a * (rbar - m->shf_a[a]) * (rbar - m->shf_a[a]));
    double fu = fc(ru, m->rc_a), fv = fc(rv, m->rc_a);
    double T = A * B * fu * fv;
    if (gu && gv) {
        double dA_dtheta = pow(2.0, 1.0 - m->zeta) * m->zeta * pow(base, m->zeta - 1.0) *
                           (-sin(theta - m->shf_z[z]));
        double dtheta_dc = -0.95 / sqrt(1.0 - 0.9025 * c * c);
        double dT_dc = dA_dtheta * dtheta_dc * B * fu * fv;
        double dB_drbar = -2.0 * m->eta_a * (rbar - m->shf_a[a]) * B;
        double dT_dru = A * (0.5 * dB_drbar * fu * fv + B * dfc(ru, m->rc_a) * fv);
        double dT_drv = A * (0.5 * dB_drbar * fu * fv + B * fu * dfc(rv, m->rc_a));
        for (int q = 0; q < 3; ++q) {
            double dc_du = dv[q] / (ru * rv) - c * du[q] / (ru * ru);
            double dc_dv = du[q] / (ru * rv) - c * dv[q] / (rv * rv);
            gu[q] = dT_dru * du[q] / ru + dT_dc * dc_du;
            gv[q] = dT_drv * dv[q] / rv + dT_dc * dc_dv;
        }
    }
    return T;
}

static int ang_index(const oracle_model *m, int sj, int sk, int a, int z) {
    int S = m->n_species;
    return m->n_rad * S + pair_index(S, sj, sk) * m->n_ang_r * m->n_ang_z + a * m->n_ang_z + z;
}

/* G_i (length D) of one atom from its radial and angular neighbour lists. */
static void aev_atom(const oracle_model *m, const int *species, const nbr_csr *rad,
                     const nbr_csr *ang, int i, double *g) {
    int D = or_aev_length(m);
    memset(g, 0, sizeof(double) * (size_t)D);
    for (long q = rad->start[i]; q < rad->start[i + 1]; ++q) {
        const double *d = rad->d + 3 * q;
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        int sj = species[rad->j[q]];
        for (int k = 0; k < m->n_rad; ++k) {
            double t, dt;
            radial_term(m, k, r, &t, &dt);
            g[sj * m->n_rad + k] += t;
        }
    }
    for (long u = ang->start[i]; u < ang->start[i + 1]; ++u)
        for (long v = u + 1; v < ang->start[i + 1]; ++v) {
            int sj = species[ang->j[u]], sk = species[ang->j[v]];
            for (int a = 0; a < m->n_ang_r; ++a)
                for (int z = 0; z < m->n_ang_z; ++z)
                    g[ang_index(m, sj, sk, a, z)] +=
                        angular_term(m, a, z, ang->d + 3 * u, ang->d + 3 * v, NULL, NULL);
        }
}

/* G (n x D) for every atom. */
static void aev_from_csr(const oracle_model *m, const int *species, const nbr_csr *rad,
                         const nbr_csr *ang, double *G) {
    int D = or_aev_length(m);
    for (int i = 0; i < rad->n; ++i) aev_atom(m, species, rad, ang, i, G + (size_t)i * D);
}

/* Adds dE_i/dr (for every atom r it depends on) to dEdr (n x 3), given
 * w = dE_i/dG_i: the chain rule of Eq. 2 through atom i's descriptor. */
static void scatter_atom(const oracle_model *m, const int *species, const nbr_csr *rad,
                         const nbr_csr *ang, int i, const double *w, double *dEdr) {
    for (long q = rad->start[i]; q < rad->start[i + 1]; ++q) {
        const double *d = rad->d + 3 * q;
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        int j = rad->j[q], sj = species[j];
        double gr = 0.0;
        for (int k = 0; k < m->n_rad; ++k) {
            double t, dt;
            radial_term(m, k, r, &t, &dt);
            gr += w[sj * m->n_rad + k] * dt;
        }
        for (int a = 0; a < 3; ++a) {
            dEdr[3 * j + a] += gr * d[a] / r;
            dEdr[3 * i + a] -= gr * d[a] / r;
        }
    }
    for (long u = ang->start[i]; u < ang->start[i + 1]; ++u)
        for (long v = u + 1; v < ang->start[i + 1]; ++v) {
            int j = ang->j[u], k = ang->j[v];
            int sj = species[j], sk = species[k];
            for (int a = 0; a < m->n_ang_r; ++a)
                for (int z = 0; z < m->n_ang_z; ++z) {
                    double gu[3], gv[3];
                    angular_term(m, a, z, ang->d + 3 * u, ang->d + 3 * v, gu, gv);
                    double wt = w[ang_index(m, sj, sk, a, z)];
                    for (int c = 0; c < 3; ++c) {
                        dEdr[3 * j + c] += wt * gu[c];
                        dEdr[3 * k + c] += wt * gv[c];
                        dEdr[3 * i + c] -= wt * (gu[c] + gv[c]);
                    }
                }
        }
}

/* AEV of every atom from a caller-supplied pair list (pairs beyond the
 * cutoffs are ignored).  G: n x D. */
int or_aev(const oracle_model *m, int n, const int *species, long np, const int *pi,
           const int *pj, const double *pd, double *G) {
    nbr_csr rad, ang;
    csr_build(&rad, n, np, pi, pj, pd, m->rc_r);
    csr_build(&ang, n, np, pi, pj, pd, m->rc_a);
    aev_from_csr(m, species, &rad, &ang, G);
    csr_free(&rad); csr_free(&ang);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* per-element MLP                                                           */

static double celu(double x, double al) { return x > 0.0 ? x : al * (exp(x / al) - 1.0); }
static double dcelu(double x, double al) { return x > 0.0 ? 1.0 : exp(x / al); }
static double d2celu(double x, double al) { return x > 0.0 ? 0.0 : exp(x / al) / al; }

#define OR_MAXW 2048

/* Forward pass of species s on one input row; returns E_i and, if dx is
 * non-NULL, dE_i/dx (the backward pass, Eq. 2's chain rule through the net). */
double or_mlp(const oracle_model *m, int s, const double *x, double *dx) {
    int L = m->n_layers;
    static OR_TLS double z[OR_MAX_LAYERS][OR_MAXW], h[OR_MAX_LAYERS + 1][OR_MAXW];
    for (int k = 0; k < m->width[0]; ++k) h[0][k] = x[k];
    for (int l = 0; l < L; ++l) {
        const double *W = m->W[s * OR_MAX_LAYERS + l], *b = m->b[s * OR_MAX_LAYERS + l];
        int fi = m->width[l], fo = m->width[l + 1];
        for (int o = 0; o < fo; ++o) {
            double acc = b[o];
            for (int k = 0; k < fi; ++k) acc += h[l][k] * W[k * fo + o];
            z[l][o] = acc;
            h[l + 1][o] = (l < L - 1) ? celu(acc, m->celu_alpha) : acc;
        }
    }
    double E = h[L][0];
    if (dx) {
        static OR_TLS double g[OR_MAXW], gn[OR_MAXW];
        g[0] = 1.0; /* dE/dz of the linear output */
        for (int l = L - 1; l >= 0; --l) {
            const double *W = m->W[s * OR_MAX_LAYERS + l];
            int fi = m->width[l], fo = m->width[l + 1];
            for (int k = 0; k < fi; ++k) {
                double acc = 0.0;
                for (int o = 0; o < fo; ++o) acc += g[o] * W[k * fo + o];
                gn[k] = acc;
            }
            if (l > 0)
                for (int k = 0; k < fi; ++k) g[k] = gn[k] * dcelu(z[l - 1][k], m->celu_alpha);
            else
                for (int k = 0; k < fi; ++k) dx[k] = gn[k];
        }
    }
    return E;
}

/* ----------------------------------------------------------------------- */
/* full energy and forces                                                    */

static long build_pairs(int n, const double *pos, const double *box, double rc,
                        int **pi, int **pj, double **pd) {
    long cap = 64;
    for (;;) {
        *pi = (int *)malloc(sizeof(int) * (size_t)cap);
        *pj = (int *)malloc(sizeof(int) * (size_t)cap);
        *pd = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
        long np = or_pairs_cells(n, pos, box, rc, cap, *pi, *pj, *pd);
        if (np <= cap) return np;
        free(*pi); free(*pj); free(*pd);
        cap = np;
    }
}

/* E (sum), Ei (n, may be NULL), F (n x 3), G (n x D, may be NULL).
 * species[i] in [0, S); box: 3 edge lengths (orthorhombic) or NULL.
 * wt (may be NULL = all ones): E = sum_i wt[i] E_i and F = -dE/dr with the
 * weights held fixed. */
static int energy_forces_from_pairs(const oracle_model *m, int n, const int *species, long np,
                                    int *pi, int *pj, double *pd, double *E, double *Ei, double *F,
                                    double *Gout, const double *wt);

int or_energy_forces(const oracle_model *m, int n, const double *pos, const int *species,
                     const double *box, double *E, double *Ei, double *F, double *Gout) {
    double rmax = m->rc_r > m->rc_a ? m->rc_r : m->rc_a;
    int *pi, *pj; double *pd;
    long np = build_pairs(n, pos, box, rmax, &pi, &pj, &pd);
    return energy_forces_from_pairs(m, n, species, np, pi, pj, pd, E, Ei, F, Gout, NULL);
}

/* As or_energy_forces with fixed per-atom weights: E = sum_i wt[i] E_i,
 * F = -dE/dr (Ei unweighted). */
int or_weighted_energy_forces(const oracle_model *m, int n, const double *pos, const int *species,
                              const double *box, const double *wt, double *E, double *Ei, double *F) {
    double rmax = m->rc_r > m->rc_a ? m->rc_r : m->rc_a;
    int *pi, *pj; double *pd;
    long np = build_pairs(n, pos, box, rmax, &pi, &pj, &pd);
    return energy_forces_from_pairs(m, n, species, np, pi, pj, pd, E, Ei, F, NULL, wt);
}

/* As or_energy_forces for a general periodic cell (rows a, b, c; pairs by
 * or_pairs_brute_cell). */
int or_energy_forces_cell(const oracle_model *m, int n, const double *pos, const int *species,
                          const double *cell, double *E, double *Ei, double *F, double *Gout) {
    double rmax = m->rc_r > m->rc_a ? m->rc_r : m->rc_a;
    long cap = 64;
    int *pi, *pj; double *pd;
    for (;;) {
        pi = (int *)malloc(sizeof(int) * (size_t)cap);
        pj = (int *)malloc(sizeof(int) * (size_t)cap);
        pd = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
        long np = or_pairs_brute_cell(n, pos, cell, rmax, cap, pi, pj, pd);
        if (np <= cap) return energy_forces_from_pairs(m, n, species, np, pi, pj, pd, E, Ei, F, Gout, NULL);
        free(pi); free(pj); free(pd);
        cap = np;
    }
}

/* E, Ei, F and G from a pair list (every ordered pair/image within the
 * largest cutoff); frees the pair arrays. */
static int energy_forces_from_pairs(const oracle_model *m, int n, const int *species, long np,
                                    int *pi, int *pj, double *pd, double *E, double *Ei, double *F,
                                    double *Gout, const double *wt) {
    int D = or_aev_length(m);
    nbr_csr rad, ang;
    csr_build(&rad, n, np, pi, pj, pd, m->rc_r);
    csr_build(&ang, n, np, pi, pj, pd, m->rc_a);
    double *G = (double *)malloc(sizeof(double) * (size_t)n * D + 8);
    double *dG = (double *)malloc(sizeof(double) * (size_t)n * D + 8);
    aev_from_csr(m, species, &rad, &ang, G);
    double Etot = 0.0;
    for (int i = 0; i < n; ++i) {
        double e = or_mlp(m, species[i], G + (size_t)i * D, dG + (size_t)i * D);
        if (Ei) Ei[i] = e;
        const double w = wt ? wt[i] : 1.0;
        if (wt)
            for (int k = 0; k < D; ++k) dG[(size_t)i * D + k] *= w;
        Etot += w * e;
    }
    *E = Etot;
    /* dE/dr by the chain rule through the AEV; F = -dE/dr */
    double *dEdr = (double *)calloc((size_t)n * 3 + 3, sizeof(double));
    for (int i = 0; i < n; ++i) scatter_atom(m, species, &rad, &ang, i, dG + (size_t)i * D, dEdr);
    for (int q = 0; q < 3 * n; ++q) F[q] = -dEdr[q];
    if (Gout) memcpy(Gout, G, sizeof(double) * (size_t)n * D);
    free(dEdr); free(G); free(dG);
    csr_free(&rad); csr_free(&ang);
    free(pi); free(pj); free(pd);
    return 0;
}

/* Sampled outputs of a large system: E_i for the atoms in sel_e and F_j for
 * the atoms in sel_f, each by the same definition as or_energy_forces.  F_j
 * needs dE_i/dr_j of every atom i that has j within its radial cutoff, so
 * those atoms (and only those) are evaluated. */
int or_energy_forces_subset(const oracle_model *m, int n, const double *pos,
                            const int *species, const double *box, int n_e, const int *sel_e,
                            double *Ei_sel, int n_f, const int *sel_f, double *F_sel) {
    int D = or_aev_length(m);
    double rmax = m->rc_r > m->rc_a ? m->rc_r : m->rc_a;
    int *pi, *pj; double *pd;
    long np = build_pairs(n, pos, box, rmax, &pi, &pj, &pd);
    nbr_csr rad, ang;
    csr_build(&rad, n, np, pi, pj, pd, m->rc_r);
    csr_build(&ang, n, np, pi, pj, pd, m->rc_a);
    double *g = (double *)malloc(sizeof(double) * (size_t)D);
    double *w = (double *)malloc(sizeof(double) * (size_t)D);
    for (int q = 0; q < n_e; ++q) {
        aev_atom(m, species, &rad, &ang, sel_e[q], g);
        Ei_sel[q] = or_mlp(m, species[sel_e[q]], g, NULL);
    }
    if (n_f > 0) {
        char *need = (char *)calloc((size_t)n, 1);
        for (int q = 0; q < n_f; ++q) {
            int j = sel_f[q];
            need[j] = 1;
            for (long t = rad.start[j]; t < rad.start[j + 1]; ++t) need[rad.j[t]] = 1;
        }
        double *dEdr = (double *)calloc((size_t)n * 3 + 3, sizeof(double));
        for (int i = 0; i < n; ++i) {
            if (!need[i]) continue;
            aev_atom(m, species, &rad, &ang, i, g);
            or_mlp(m, species[i], g, w);
            scatter_atom(m, species, &rad, &ang, i, w, dEdr);
        }
        for (int q = 0; q < n_f; ++q)
            for (int c = 0; c < 3; ++c) F_sel[3 * q + c] = -dEdr[3 * sel_f[q] + c];
        free(need); free(dEdr);
    }
    free(g); free(w);
    csr_free(&rad); csr_free(&ang);
    free(pi); free(pj); free(pd);
    return 0;
}

/* Directional derivative of every atom's AEV along per-atom displacements
 * v (n x 3): dG_i = sum_j (dG_i/dr_j) . v_j.  dGout: n x D. */
int or_aev_jvp(const oracle_model *m, int n, const double *pos, const int *species,
               const double *box, const double *v, double *dGout) {
    int D = or_aev_length(m);
    double rmax = m->rc_r > m->rc_a ? m->rc_r : m->rc_a;
    int *pi, *pj; double *pd;
    long np = build_pairs(n, pos, box, rmax, &pi, &pj, &pd);
    nbr_csr rad, ang;
    csr_build(&rad, n, np, pi, pj, pd, m->rc_r);
    csr_build(&ang, n, np, pi, pj, pd, m->rc_a);
    memset(dGout, 0, sizeof(double) * (size_t)n * D);
    for (int i = 0; i < n; ++i) {
        double *t = dGout + (size_t)i * D;
        for (long q = rad.start[i]; q < rad.start[i + 1]; ++q) {
            const double *d = rad.d + 3 * q;
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            int j = rad.j[q], sj = species[j];
            double dr = 0.0; /* d r_ij along v */
            for (int a = 0; a < 3; ++a) dr += d[a] / r * (v[3 * j + a] - v[3 * i + a]);
            for (int k = 0; k < m->n_rad; ++k) {
                double tt, dt;
                radial_term(m, k, r, &tt, &dt);
                t[sj * m->n_rad + k] += dt * dr;
            }
        }
        for (long u = ang.start[i]; u < ang.start[i + 1]; ++u)
            for (long w = u + 1; w < ang.start[i + 1]; ++w) {
                int j = ang.j[u], k = ang.j[w];
                int sj = species[j], sk = species[k];
                for (int a = 0; a < m->n_ang_r; ++a)
                    for (int z = 0; z < m->n_ang_z; ++z) {
                        double gu[3], gv[3];
                        angular_term(m, a, z, ang.d + 3 * u, ang.d + 3 * w, gu, gv);
                        double s = 0.0;
                        for (int c = 0; c < 3; ++c)
                            s += gu[c] * (v[3 * j + c] - v[3 * i + c]) +
                                 gv[c] * (v[3 * k + c] - v[3 * i + c]);
                        t[ang_index(m, sj, sk, a, z)] += s;
                    }
            }
    }
    csr_free(&rad); csr_free(&ang);
    free(pi); free(pj); free(pd);
    return 0;
}

/* Force-matching loss L = 1/(3N) sum |F - Fref|^2 and its weight gradients.
 * dW[s*OR_MAX_LAYERS + l], db[...] point to caller buffers shaped like W, b
 * (overwritten).  Fout (n x 3, may be NULL) receives F. */
int or_force_match(const oracle_model *m, int n, const double *pos, const int *species,
                   const double *box, const double *Fref, double *Lout,
                   double *const *dW, double *const *db, double *Fout) {
    int D = or_aev_length(m);
    int L = m->n_layers;
    double E;
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)n + 8);
    double *G = (double *)malloc(sizeof(double) * (size_t)n * D + 8);
    or_energy_forces(m, n, pos, species, box, &E, NULL, F, G);
    double loss = 0.0;
    double *v = (double *)malloc(sizeof(double) * 3 * (size_t)n + 8);
    for (int q = 0; q < 3 * n; ++q) {
        double e = F[q] - Fref[q];
        loss += e * e;
        v[q] = 2.0 * e / (3.0 * n);         /* v = dL/dF */
    }
    *Lout = loss / (3.0 * n);
    if (Fout) memcpy(Fout, F, sizeof(double) * 3 * (size_t)n);
    double *T = (double *)malloc(sizeof(double) * (size_t)n * D + 8);
    or_aev_jvp(m, n, pos, species, box, v, T);  /* dG along v */
    for (int s = 0; s < m->n_species; ++s)
        for (int l = 0; l < L; ++l) {
            memset(dW[s * OR_MAX_LAYERS + l], 0, sizeof(double) * m->width[l] * m->width[l + 1]);
            memset(db[s * OR_MAX_LAYERS + l], 0, sizeof(double) * m->width[l + 1]);
        }
    /* per atom: phi = <dE_i/dG_i, dG_i> is the tangent of E_i along dG_i;
     * dL/dtheta = -sum_i dphi_i/dtheta (reverse pass over the tangent pass). */
    static double z[OR_MAX_LAYERS][OR_MAXW], h[OR_MAX_LAYERS + 1][OR_MAXW];
    static double dz[OR_MAX_LAYERS][OR_MAXW], dh[OR_MAX_LAYERS + 1][OR_MAXW];
    static double th[OR_MAXW], ph[OR_MAXW], tz[OR_MAXW], pz[OR_MAXW], tn[OR_MAXW], pn[OR_MAXW];
    for (int i = 0; i < n; ++i) {
        int s = species[i];
        for (int k = 0; k < D; ++k) { h[0][k] = G[(size_t)i * D + k]; dh[0][k] = T[(size_t)i * D + k]; }
        for (int l = 0; l < L; ++l) {
            const double *W = m->W[s * OR_MAX_LAYERS + l], *b = m->b[s * OR_MAX_LAYERS + l];
            int fi = m->width[l], fo = m->width[l + 1];
            for (int o = 0; o < fo; ++o) {
                double acc = b[o], tac = 0.0;
                for (int k = 0; k < fi; ++k) { acc += h[l][k] * W[k * fo + o]; tac += dh[l][k] * W[k * fo + o]; }
                z[l][o] = acc; dz[l][o] = tac;
                if (l < L - 1) {
                    h[l + 1][o] = celu(acc, m->celu_alpha);
                    dh[l + 1][o] = dcelu(acc, m->celu_alpha) * tac;
                } else { h[l + 1][o] = acc; dh[l + 1][o] = tac; }
            }
        }
        /* reverse: output layer is linear, phi = dz[L-1][0] */
        for (int l = L - 1; l >= 0; --l) {
            int fi = m->width[l], fo = m->width[l + 1];
            const double *W = m->W[s * OR_MAX_LAYERS + l];
            double *gW = dW[s * OR_MAX_LAYERS + l], *gb = db[s * OR_MAX_LAYERS + l];
            if (l == L - 1) {
                for (int o = 0; o < fo; ++o) { tz[o] = 1.0; pz[o] = 0.0; }
            } else {
                for (int o = 0; o < fo; ++o) {
                    double sp = dcelu(z[l][o], m->celu_alpha);
                    double spp = d2celu(z[l][o], m->celu_alpha);
                    tz[o] = sp * th[o];
                    pz[o] = sp * ph[o] + spp * dz[l][o] * th[o];
                }
            }
            for (int k = 0; k < fi; ++k)
                for (int o = 0; o < fo; ++o)
                    gW[k * fo + o] -= dh[l][k] * tz[o] + h[l][k] * pz[o];
            for (int o = 0; o < fo; ++o) gb[o] -= pz[o];
            if (l > 0) {
                for (int k = 0; k < fi; ++k) {
                    double a1 = 0.0, a2 = 0.0;
                    for (int o = 0; o < fo; ++o) { a1 += tz[o] * W[k * fo + o]; a2 += pz[o] * W[k * fo + o]; }
                    tn[k] = a1; pn[k] = a2;
                }
                for (int k = 0; k < fi; ++k) { th[k] = tn[k]; ph[k] = pn[k]; }
            }
        }
    }
    free(F); free(G); free(v); free(T);
    return 0;
}
