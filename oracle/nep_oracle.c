/*
 * nep_oracle.c -- plain, slow FP64 CPU oracle of the NEP-ZBL potential
 * (Sec. II.A, Eq. 1-4) and of velocity-Verlet MD (Sec. II.B).
 *
 * TEST INFRASTRUCTURE ONLY.  It is used by the tests, by the bench's CPU
 * baseline and by the scaler script; the product (the CUDA library) never
 * calls, links or includes it, and it shares no code with it.
 *
 * What it computes, written out from the definitions:
 *   E = sum_i U_i,  U_i = U_i^NEP({q_nu^i}) + 1/2 sum_{j != i} U_ZBL(r_ij)   (Eq. 1)
 *   U_ZBL(r) = e^2/(4 pi eps0) Zi Zj / r * phi(r/a) * f_c(r)                  (Eq. 2)
 *   phi(x) = 0.32825 e^{-2.54931 x} + 0.09219 e^{-0.29182 x}
 *            + 0.58110 e^{-0.59231 x}                                         (Eq. 3)
 *   a = 0.46848 / (Zi^0.23 + Zj^0.23)                                         (Eq. 4)
 *   f_c = Tersoff switch with inner 1.0 A and outer 2.0 A                     (Sec. II.A)
 * The NEP site energy is a one-hidden-layer tanh network (Behler-Parrinello,
 * Sec. II.A) of a descriptor with Chebyshev radial and Legendre angular parts
 * (Sec. II.A).  The paper defers the exact descriptor to the NEP papers it
 * cites; the reading used here (same as the CUDA path's contract):
 *   f_c(r; rc)  = (1 + cos(pi r / rc)) / 2 for r < rc, else 0
 *   f_k(r; rc)  = (T_k(x) + 1)/2 * f_c(r; rc),  x = 2 (r/rc - 1)^2 - 1, k = 0..K-1
 *   g_n(r)      = sum_k c_nk f_k(r)       (separate c for radial / angular)
 *   q_n         = sum_j g^R_n(r_ij)                                 n = 0..nR-1
 *   q_nl        = sum_j sum_k g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_ijk)
 *                 (j = k included), l = 1..lmax, stored l-major
 *   q^4b_n      = tr(T_n^3), T_n = sum_j g^A_n(r_ij) (u_ij u_ij^T - I/3)
 *   U^NEP       = sum_mu w1_mu tanh(sum_nu w0_{mu nu} s_nu q_nu - b0_mu) - b1
 * With several species (T types) every pair term uses the coefficients of
 * its ordered species pair: g_n of the pair (i, j) is sum_k c^{t_i t_j}_nk
 * f_k(r_ij), t_i the species of the centre, t_j of the neighbour; the network
 * is shared by all species; Z_i, Z_j in Eq. 2 and 4 are the pair's charges.
 * Forces are F = -dE/dr, virial W_ab = -sum_i sum_j (dU_i/dr_ij)_a (r_ij)_b,
 * with r_ij = r_j - r_i, all from analytic FP64 derivatives of the formulas
 * above (the Legendre double sum and the 3x3 tensor form, not spherical
 * harmonics).
 *
 * Neighbours: either brute force over all atoms and all periodic images
 * (self-images included), or a plain cell grid with the minimum image (only
 * when every periodic box length holds at least three cells of size >= rc).
 *
 * Cells: box = 9 doubles, the rows of H are the cell vectors a, b, c, and a
 * position is x = s H with fractional s (periodic dimensions wrap s into
 * [0, 1)).  A diagonal H is the orthorhombic box of lengths H_aa; any other
 * (triclinic) H uses brute-force neighbours with images x_j - x_i + n H.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_MEM (-2)
#define ORC_MAX_TYPES 8

/* e^2 / (4 pi eps0) in eV*A (CODATA), the prefactor of Eq. 2 */
#define ORC_COULOMB 14.39964547
/* 1 eV/amu in A^2/fs^2 (CODATA e and u) */
#define ORC_EV_AMU (1.602176634e-19 / 1.66053906660e-27 * 1e-10)

typedef struct {
    double rcR, rcA;     /* radial / angular cutoff (A) */
    int nR, nA;          /* number of radial / angular functions g_n */
    int KR, KA;          /* number of Chebyshev basis functions */
    int lmax;            /* angular orders l = 1..lmax */
    int use4b;           /* 4-body term on/off */
    int H;               /* hidden neurons */
    int D;               /* descriptor length */
    int T;               /* number of species */
    double Z[ORC_MAX_TYPES];  /* nuclear charge per species */
    double zr1, zr2;     /* Tersoff switch radii of the ZBL term */
    const double *w0, *b0, *w1, *b1;  /* views into params */
    const double *cR, *cA;   /* [T][T][n][K]: block (t_i, t_j) */
    const double *s;     /* descriptor scaler, length D */
} orc_model;

/* Radial / angular coefficients c^{ti tj} of an ordered species pair. */
static const double *coef_R(const orc_model *m, int ti, int tj)
{
    return m->cR + (size_t)(ti * m->T + tj) * m->nR * m->KR;
}
static const double *coef_A(const orc_model *m, int ti, int tj)
{
    return m->cA + (size_t)(ti * m->T + tj) * m->nA * m->KA;
}

/* ihp = {nR, nA, KR, KA, lmax, use4b, H, T};
 * dhp = {rcR, rcA, zr1, zr2, Z_0, ..., Z_{T-1}};
 * params = w0[H][D], b0[H], w1[H], b1, cR[T][T][nR][KR], cA[T][T][nA][KA] */
static int model_init(orc_model *m, const int *ihp, const double *dhp,
                      const double *params, const double *scaler)
{
    m->nR = ihp[0]; m->nA = ihp[1]; m->KR = ihp[2]; m->KA = ihp[3];
    m->lmax = ihp[4]; m->use4b = ihp[5]; m->H = ihp[6]; m->T = ihp[7];
    m->rcR = dhp[0]; m->rcA = dhp[1]; m->zr1 = dhp[2]; m->zr2 = dhp[3];
    if (m->nR < 1 || m->nA < 1 || m->nA > 16 || m->nR > 64 || m->KR < 1 ||
        m->KA < 1 || m->KR > 64 || m->KA > 64 || m->lmax < 0 || m->lmax > 63 ||
        m->H < 1 || !(m->rcR > 0) || !(m->rcA > 0) || !(m->zr2 > m->zr1) ||
        m->T < 1 || m->T > ORC_MAX_TYPES)
        return ORC_ERR_ARG;
    for (int t = 0; t < m->T; ++t) {
        m->Z[t] = dhp[4 + t];
        if (!(m->Z[t] > 0)) return ORC_ERR_ARG;
    }
    m->D = m->nR + m->nA * m->lmax + (m->use4b ? m->nA : 0);
    const double *p = params;
    m->w0 = p; p += (size_t)m->H * m->D;
    m->b0 = p; p += m->H;
    m->w1 = p; p += m->H;
    m->b1 = p; p += 1;
    m->cR = p; p += (size_t)m->T * m->T * m->nR * m->KR;
    m->cA = p;
    m->s = scaler;
    return ORC_OK;
}

int orc_n_params(const int *ihp)
{
    int nR = ihp[0], nA = ihp[1], KR = ihp[2], KA = ihp[3], lmax = ihp[4];
    int use4b = ihp[5], H = ihp[6], T = ihp[7];
    int D = nR + nA * lmax + (use4b ? nA : 0);
    return H * D + 2 * H + 1 + T * T * (nR * KR + nA * KA);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * One-dimensional building blocks
 * ------------------------------------------------------------------------- */

/* Smooth cutoff (1 + cos(pi r/rc))/2 and its r-derivative. */
void orc_cutoff(double r, double rc, double *fc, double *dfc)
{
    if (r < rc) {
        *fc = 0.5 * (1.0 + cos(M_PI * r / rc));
        *dfc = -0.5 * M_PI / rc * sin(M_PI * r / rc);
    } else {
        *fc = 0.0;
        *dfc = 0.0;
    }
}

/* Chebyshev polynomials of the first kind T_0..T_{K-1} at x and dT_k/dx,
 * from T_{k+1} = 2x T_k - T_{k-1} and its derivative. */
void orc_chebyshev(double x, int K, double *T, double *dT)
{
    for (int k = 0; k < K; ++k) {
        if (k == 0) { T[0] = 1.0; dT[0] = 0.0; }
        else if (k == 1) { T[1] = x; dT[1] = 1.0; }
        else {
            T[k] = 2.0 * x * T[k - 1] - T[k - 2];
            dT[k] = 2.0 * T[k - 1] + 2.0 * x * dT[k - 1] - dT[k - 2];
        }
    }
}

/* Basis f_k(r) = (T_k(x) + 1)/2 * f_c(r), x = 2 (r/rc - 1)^2 - 1, and df_k/dr. */
void orc_basis(double r, double rc, int K, double *f, double *df)
{
    double fc, dfc;
    orc_cutoff(r, rc, &fc, &dfc);
    double t = r / rc - 1.0;
    double x = 2.0 * t * t - 1.0;
    double dxdr = 4.0 * t / rc;
    double T[64], dT[64];
    orc_chebyshev(x, K, T, dT);
    for (int k = 0; k < K; ++k) {
        f[k] = 0.5 * (T[k] + 1.0) * fc;
        df[k] = 0.5 * dT[k] * dxdr * fc + 0.5 * (T[k] + 1.0) * dfc;
    }
}

/* g_n(r) = sum_k c[n][k] f_k(r) and dg_n/dr for n = 0..nn-1. */
static void radial_functions(const double *c, int nn, int K, double r, double rc,
                             double *g, double *dg)
{
    double f[64], df[64];
    orc_basis(r, rc, K, f, df);
    for (int n = 0; n < nn; ++n) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < K; ++k) {
            a += c[n * K + k] * f[k];
            b += c[n * K + k] * df[k];
        }
        g[n] = a;
        dg[n] = b;
    }
}

/* Legendre polynomials P_0..P_lmax at x and their derivatives, from
 * (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1} and P'_{l+1} = P'_{l-1} + (2l+1) P_l. */
void orc_legendre(double x, int lmax, double *P, double *dP)
{
    for (int l = 0; l <= lmax; ++l) {
        if (l == 0) { P[0] = 1.0; dP[0] = 0.0; }
        else if (l == 1) { P[1] = x; dP[1] = 1.0; }
        else {
            P[l] = ((2.0 * l - 1.0) * x * P[l - 1] - (l - 1.0) * P[l - 2]) / l;
            dP[l] = dP[l - 2] + (2.0 * l - 1.0) * P[l - 1];
        }
    }
}

/* ZBL-like W-W repulsion, Eq. 2-4, times the Tersoff switch (inner r1, outer
 * r2).  Returns U(r) and dU/dr. */
void orc_zbl(double r, double Zi, double Zj, double r1, double r2,
             double *U, double *dU)
{
    if (!(r < r2)) { *U = 0.0; *dU = 0.0; return; }
    double a = 0.46848 / (pow(Zi, 0.23) + pow(Zj, 0.23));
    static const double c[3] = {0.32825, 0.09219, 0.58110};
    static const double b[3] = {2.54931, 0.29182, 0.59231};
    double x = r / a;
    double phi = 0.0, dphi = 0.0;   /* dphi = d phi / dx */
    for (int i = 0; i < 3; ++i) {
        double e = c[i] * exp(-b[i] * x);
        phi += e;
        dphi -= b[i] * e;
    }
    double fc, dfc;
    if (r < r1) { fc = 1.0; dfc = 0.0; }
    else {
        double arg = M_PI * (r - r1) / (r2 - r1);
        fc = 0.5 + 0.5 * cos(arg);
        dfc = -0.5 * M_PI / (r2 - r1) * sin(arg);
    }
    double k = ORC_COULOMB * Zi * Zj;
    double v = k / r * phi;                                   /* unswitched */
    double dv = -k / (r * r) * phi + k / r * dphi / a;
    *U = v * fc;
    *dU = dv * fc + v * dfc;
}

/* ---------------------------------------------------------------------------
 * NEP site energy of one atom
 * ------------------------------------------------------------------------- */

/* Descriptor q (length D) of one atom of species ti from the displacement
 * vectors of its radial neighbours dR[3*nr] (r < rcR, species tR[nr]) and
 * angular neighbours dA[3*na] (r < rcA, species tA[na]).  If the gradient
 * buffers are given, also returns dU^NEP/dd for each neighbour (gR[3*nr],
 * gA[3*na]) and U^NEP itself. */
static double site_nep(const orc_model *m, int ti, int nr, const double *dR, const int *tR,
                       int na, const double *dA, const int *tA, double *q_out, double *gR,
                       double *gA, double *cond)
{
    const int nR = m->nR, nA = m->nA, L = m->lmax, D = m->D, H = m->H;
    double *q = (double *)calloc((size_t)D, sizeof(double));
    double *rA = (double *)malloc(sizeof(double) * (size_t)(na > 0 ? na : 1));
    double *uA = (double *)malloc(sizeof(double) * 3 * (size_t)(na > 0 ? na : 1));
    double *gnA = (double *)malloc(sizeof(double) * (size_t)nA * (na > 0 ? na : 1));
    double *dgnA = (double *)malloc(sizeof(double) * (size_t)nA * (na > 0 ? na : 1));
    double g[64], dg[64];

    /* radial part: q_n = sum_j g^R_n(r_ij) */
    for (int s = 0; s < nr; ++s) {
        const double *d = dR + 3 * s;
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        radial_functions(coef_R(m, ti, tR[s]), nR, m->KR, r, m->rcR, g, dg);
        for (int n = 0; n < nR; ++n) q[n] += g[n];
    }
    /* angular neighbours: distance, unit vector, g^A_n and dg^A_n/dr */
    for (int s = 0; s < na; ++s) {
        const double *d = dA + 3 * s;
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        rA[s] = r;
        for (int a = 0; a < 3; ++a) uA[3 * s + a] = d[a] / r;
        radial_functions(coef_A(m, ti, tA[s]), nA, m->KA, r, m->rcA, g, dg);
        for (int n = 0; n < nA; ++n) { gnA[n * na + s] = g[n]; dgnA[n * na + s] = dg[n]; }
    }
    /* q_nl: Legendre double sum over all ordered pairs (j, k), j = k included */
    double P[64], dP[64];
    for (int s = 0; s < na; ++s)
        for (int t = 0; t < na; ++t) {
            double c = uA[3 * s] * uA[3 * t] + uA[3 * s + 1] * uA[3 * t + 1] +
                       uA[3 * s + 2] * uA[3 * t + 2];
            orc_legendre(c, L, P, dP);
            for (int l = 1; l <= L; ++l)
                for (int n = 0; n < nA; ++n)
                    q[nR + (l - 1) * nA + n] += gnA[n * na + s] * gnA[n * na + t] * P[l];
        }
    /* 4-body: T_n = sum_j g^A_n (u u^T - I/3); q = tr(T^3) */
    double T[16][3][3];
    if (m->use4b) {
        for (int n = 0; n < nA; ++n) {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double acc = 0.0;
                    for (int s = 0; s < na; ++s)
                        acc += gnA[n * na + s] *
                               (uA[3 * s + a] * uA[3 * s + b] - (a == b ? 1.0 / 3.0 : 0.0));
                    T[n][a][b] = acc;
                }
            double tr3 = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    for (int c = 0; c < 3; ++c)
                        tr3 += T[n][a][b] * T[n][b][c] * T[n][c][a];
            q[nR + L * nA + n] = tr3;
        }
    }
    if (q_out) memcpy(q_out, q, sizeof(double) * (size_t)D);

    /* network: U = sum_mu w1_mu tanh(sum_nu w0_{mu nu} s_nu q_nu - b0_mu) - b1 */
    double U = -m->b1[0];
    double *dUdq = (double *)calloc((size_t)D, sizeof(double));
    double hmax = 0.0, nsens = 0.0, tmag = fabs(m->b1[0]);
    for (int mu = 0; mu < H; ++mu) {
        double h = -m->b0[mu], habs = 0.0;
        for (int nu = 0; nu < D; ++nu) {
            h += m->w0[mu * D + nu] * m->s[nu] * q[nu];
            habs += fabs(m->w0[mu * D + nu] * m->s[nu] * q[nu]);
        }
        double th = tanh(h);
        U += m->w1[mu] * th;
        double back = m->w1[mu] * (1.0 - th * th);
        for (int nu = 0; nu < D; ++nu) dUdq[nu] += back * m->w0[mu * D + nu] * m->s[nu];
        if (habs > hmax) hmax = habs;
        nsens += fabs(back) * habs;
        tmag += fabs(m->w1[mu] * th);
    }
    /* conditioning of the site (test support, for rounding-error bounds):
     * radial neighbour count, max_mu sum_nu |w0 s q| (the scale of the
     * pre-activations' rounding), sum_mu |w1 (1 - t^2)| sum_nu |w0 s q| (the
     * sensitivity of U to relative descriptor errors) and sum |terms of U| */
    if (cond) {
        cond[0] = (double)nr;
        cond[1] = hmax;
        cond[2] = nsens;
        cond[3] = tmag;
    }

    if (gR) {
        for (int s = 0; s < nr; ++s) {
            const double *d = dR + 3 * s;
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            radial_functions(coef_R(m, ti, tR[s]), nR, m->KR, r, m->rcR, g, dg);
            double sc = 0.0;
            for (int n = 0; n < nR; ++n) sc += dUdq[n] * dg[n];
            for (int a = 0; a < 3; ++a) gR[3 * s + a] = sc * d[a] / r;
        }
    }
    if (gA) {
        for (int s = 0; s < na; ++s) {
            double grad[3] = {0.0, 0.0, 0.0};
            const double *us = uA + 3 * s;
            double rs = rA[s];
            /* d q_nl / d d_s = 2 sum_t g_t [g'_s P_l(c_st) u_s + g_s P_l'(c_st) (u_t - c_st u_s)/r_s] */
            for (int t = 0; t < na; ++t) {
                const double *ut = uA + 3 * t;
                double c = us[0] * ut[0] + us[1] * ut[1] + us[2] * ut[2];
                orc_legendre(c, L, P, dP);
                for (int l = 1; l <= L; ++l)
                    for (int n = 0; n < nA; ++n) {
                        double w = dUdq[nR + (l - 1) * nA + n];
                        double gs = gnA[n * na + s], gt = gnA[n * na + t];
                        double dgs = dgnA[n * na + s];
                        for (int a = 0; a < 3; ++a)
                            grad[a] += w * 2.0 * gt *
                                       (dgs * P[l] * us[a] + gs * dP[l] * (ut[a] - c * us[a]) / rs);
                    }
            }
            /* d tr(T^3)/d d_s = 3 sum_{ab} (T^2)_{ba} dT_ab/dd_s with
             * dT_ab/dd_e = g' u_e Q_ab + g (d_ae u_b + u_a d_be - 2 u_a u_b u_e)/r */
            if (m->use4b) {
                for (int n = 0; n < nA; ++n) {
                    double w = dUdq[nR + L * nA + n];
                    double T2[3][3];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) {
                            double acc = 0.0;
                            for (int c = 0; c < 3; ++c) acc += T[n][a][c] * T[n][c][b];
                            T2[a][b] = acc;
                        }
                    double gs = gnA[n * na + s], dgs = dgnA[n * na + s];
                    for (int e = 0; e < 3; ++e) {
                        double acc = 0.0;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                double Qab = us[a] * us[b] - (a == b ? 1.0 / 3.0 : 0.0);
                                double dQ = ((a == e ? us[b] : 0.0) + (b == e ? us[a] : 0.0) -
                                             2.0 * us[a] * us[b] * us[e]) / rs;
                                acc += 3.0 * T2[b][a] * (dgs * us[e] * Qab + gs * dQ);
                            }
                        grad[e] += w * acc;
                    }
                }
            }
            for (int a = 0; a < 3; ++a) gA[3 * s + a] = grad[a];
        }
    }
    free(q); free(rA); free(uA); free(gnA); free(dgnA); free(dUdq);
    return U;
}

/* Exported single-environment evaluation (for tests): U^NEP, q and gradients
 * of one atom given its neighbour displacements. */
int orc_site(const int *ihp, const double *dhp, const double *params,
             const double *scaler, int ti, int nr, const double *dR, const int *tR, int na,
             const double *dA, const int *tA, double *U, double *q, double *gR, double *gA)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler)) return ORC_ERR_ARG;
    if (ti < 0 || ti >= m.T) return ORC_ERR_ARG;
    for (int s = 0; s < nr; ++s) if (tR[s] < 0 || tR[s] >= m.T) return ORC_ERR_ARG;
    for (int s = 0; s < na; ++s) if (tA[s] < 0 || tA[s] >= m.T) return ORC_ERR_ARG;
    *U = site_nep(&m, ti, nr, dR, tR, na, dA, tA, q, gR, gA, NULL);
    return ORC_OK;
}

/* 4-body invariant by the triple sum sum_{jkl} g_j g_k g_l tr(Q_j Q_k Q_l),
 * Q = u u^T - I/3 (for tests of the tensor form on tiny environments). */
double orc_fourbody_triple(int na, const double *g, const double *u)
{
    double tot = 0.0;
    for (int j = 0; j < na; ++j)
        for (int k = 0; k < na; ++k)
            for (int l = 0; l < na; ++l) {
                double Q[3][3][3];
                const int id[3] = {j, k, l};
                for (int t = 0; t < 3; ++t)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            Q[t][a][b] = u[3 * id[t] + a] * u[3 * id[t] + b] -
                                         (a == b ? 1.0 / 3.0 : 0.0);
                double tr = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        for (int c = 0; c < 3; ++c) tr += Q[0][a][b] * Q[1][b][c] * Q[2][c][a];
                tot += g[j] * g[k] * g[l] * tr;
            }
    return tot;
}

/* ---------------------------------------------------------------------------
 * Neighbours
 * ------------------------------------------------------------------------- */

typedef struct {
    int n, cap;
    int *j;        /* neighbour atom */
    int *t;        /* its species */
    double *d;     /* displacement r_j (+ image) - r_i, 3 per entry */
    double *g;     /* dU_i/dd for this entry, 3 per entry */
} orc_list;

static int list_push(orc_list *L, int j, int t, const double *d)
{
    if (L->n == L->cap) {
        int cap = L->cap ? 2 * L->cap : 32;
        int *nj = (int *)realloc(L->j, sizeof(int) * (size_t)cap);
        if (!nj) return ORC_ERR_MEM;
        L->j = nj;
        int *nt = (int *)realloc(L->t, sizeof(int) * (size_t)cap);
        if (!nt) return ORC_ERR_MEM;
        L->t = nt;
        double *nd = (double *)realloc(L->d, sizeof(double) * 3 * (size_t)cap);
        if (!nd) return ORC_ERR_MEM;
        L->d = nd;
        L->cap = cap;
    }
    L->j[L->n] = j;
    L->t[L->n] = t;
    for (int a = 0; a < 3; ++a) L->d[3 * L->n + a] = d[a];
    L->n++;
    return ORC_OK;
}

static void list_free(orc_list *L)
{
    free(L->j); free(L->t); free(L->d); free(L->g);
    memset(L, 0, sizeof(*L));
}

typedef struct {
    int N;
    const double *pos;   /* (N,3) */
    double box[3];       /* diagonal of H */
    int pbc[3];
    const int *types;    /* (N) species, or NULL for all 0 */
    int tric;            /* H has off-diagonal entries */
    double h[9], hinv[9];   /* H (rows a, b, c) and its inverse */
} orc_sys;

static int sys_type(const orc_sys *S, int i) { return S->types ? S->types[i] : 0; }

/* Fills the cell of S from the row-major 3x3 H; 0 if det H <= 0. */
static int sys_cell(orc_sys *S, const double *h)
{
    memcpy(S->h, h, sizeof(S->h));
    S->tric = 0;
    for (int a = 0; a < 3; ++a) {
        S->box[a] = h[4 * a];
        for (int b = 0; b < 3; ++b)
            if (a != b && h[3 * a + b] != 0.0) S->tric = 1;
    }
    const double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8],
                 c02 = h[3] * h[7] - h[4] * h[6];
    const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (!(det > 0)) return 0;
    /* inverse = adjugate / det */
    S->hinv[0] = c00 / det;
    S->hinv[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    S->hinv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    S->hinv[3] = c01 / det;
    S->hinv[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    S->hinv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    S->hinv[6] = c02 / det;
    S->hinv[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    S->hinv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    return 1;
}

/* Fractional coordinates s = x H^-1 (row vectors). */
static void to_frac(const orc_sys *S, const double *x, double *f)
{
    for (int a = 0; a < 3; ++a)
        f[a] = x[0] * S->hinv[a] + x[1] * S->hinv[3 + a] + x[2] * S->hinv[6 + a];
}

/* Perpendicular width of the cell along lattice direction a: V / |b x c|. */
static double cell_width(const orc_sys *S, int a)
{
    const double *u = S->h + 3 * ((a + 1) % 3), *v = S->h + 3 * ((a + 2) % 3);
    const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
                 cz = u[0] * v[1] - u[1] * v[0];
    const double *w = S->h + 3 * a;
    return fabs(w[0] * cx + w[1] * cy + w[2] * cz) / sqrt(cx * cx + cy * cy + cz * cz);
}

/* Periodic wrap of one position (triclinic): x -= sum_a floor(s_a) H_a. */
static void wrap_tric(const orc_sys *S, double *x)
{
    double f[3];
    to_frac(S, x, f);
    for (int a = 0; a < 3; ++a) {
        if (!S->pbc[a]) continue;
        const double k = floor(f[a]);
        if (k != 0.0)
            for (int b = 0; b < 3; ++b) x[b] -= k * S->h[3 * a + b];
    }
}

/* Every species index in [0, T). */
static int types_valid(const orc_sys *S, int T)
{
    if (!S->types) return 1;
    for (int i = 0; i < S->N; ++i)
        if (S->types[i] < 0 || S->types[i] >= T) return 0;
    return 1;
}

typedef struct {
    int use;             /* 0: brute force */
    int nc[3];
    double lo[3], lc[3];
    int *head, *next;
} orc_grid;

/* Brute force: every atom j and every periodic image with |d| < rc, the atom
 * itself excluded only at zero shift. */
static int query_brute_tric(const orc_sys *S, int i, double rc, orc_list *out)
{
    int nmax[3];
    for (int a = 0; a < 3; ++a)
        nmax[a] = S->pbc[a] ? (int)ceil(rc / cell_width(S, a)) + 1 : 0;
    const double *xi = S->pos + 3 * i;
    double rc2 = rc * rc;
    for (int j = 0; j < S->N; ++j) {
        const double *xj = S->pos + 3 * j;
        double base[3], f[3];
        for (int a = 0; a < 3; ++a) base[a] = xj[a] - xi[a];
        to_frac(S, base, f);
        for (int a = 0; a < 3; ++a) {
            if (!S->pbc[a]) continue;
            const double k = floor(f[a] + 0.5);
            for (int b = 0; b < 3; ++b) base[b] -= k * S->h[3 * a + b];
        }
        for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
            for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                    double d[3];
                    for (int b = 0; b < 3; ++b)
                        d[b] = base[b] + n0 * S->h[b] + n1 * S->h[3 + b] + n2 * S->h[6 + b];
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
                    if (r2 < rc2 && list_push(out, j, sys_type(S, j), d)) return ORC_ERR_MEM;
                }
    }
    return ORC_OK;
}

static int query_brute(const orc_sys *S, int i, double rc, orc_list *out)
{
    if (S->tric) return query_brute_tric(S, i, rc, out);
    int nmax[3];
    for (int a = 0; a < 3; ++a)
        nmax[a] = S->pbc[a] ? (int)ceil(rc / S->box[a]) + 1 : 0;
    const double *xi = S->pos + 3 * i;
    double rc2 = rc * rc;
    for (int j = 0; j < S->N; ++j) {
        const double *xj = S->pos + 3 * j;
        double base[3];
        for (int a = 0; a < 3; ++a) {
            base[a] = xj[a] - xi[a];
            if (S->pbc[a]) base[a] -= S->box[a] * floor(base[a] / S->box[a] + 0.5);
        }
        for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
            for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                    double d[3] = {base[0] + n0 * S->box[0], base[1] + n1 * S->box[1],
                                   base[2] + n2 * S->box[2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
                    if (r2 < rc2 && list_push(out, j, sys_type(S, j), d)) return ORC_ERR_MEM;
                }
    }
    return ORC_OK;
}

/* Cell grid with cells of at least rc; usable when every periodic dimension
 * has >= 3 cells (then the minimum image is the only image within rc). */
static int grid_build(const orc_sys *S, double rc, orc_grid *G)
{
    memset(G, 0, sizeof(*G));
    if (S->tric) return ORC_OK;                   /* brute force */
    for (int a = 0; a < 3; ++a) {
        if (S->pbc[a]) {
            int nc = (int)floor(S->box[a] / rc);
            if (nc < 3) return ORC_OK;            /* brute force */
            G->nc[a] = nc; G->lo[a] = 0.0; G->lc[a] = S->box[a] / nc;
        } else {
            double lo = 1e300, hi = -1e300;
            for (int i = 0; i < S->N; ++i) {
                double x = S->pos[3 * i + a];
                if (x < lo) lo = x;
                if (x > hi) hi = x;
            }
            if (S->N == 0) { lo = 0; hi = 0; }
            int nc = (int)floor((hi - lo) / rc);
            if (nc < 1) nc = 1;
            G->nc[a] = nc; G->lo[a] = lo; G->lc[a] = (hi - lo) / nc;
            if (!(G->lc[a] > 0)) G->lc[a] = rc;
        }
    }
    size_t ncell = (size_t)G->nc[0] * G->nc[1] * G->nc[2];
    G->head = (int *)malloc(sizeof(int) * ncell);
    G->next = (int *)malloc(sizeof(int) * (size_t)(S->N > 0 ? S->N : 1));
    if (!G->head || !G->next) return ORC_ERR_MEM;
    for (size_t c = 0; c < ncell; ++c) G->head[c] = -1;
    for (int i = S->N - 1; i >= 0; --i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double x = S->pos[3 * i + a];
            if (S->pbc[a]) x -= S->box[a] * floor(x / S->box[a]);
            int k = (int)floor((x - G->lo[a]) / G->lc[a]);
            if (k < 0) k = 0;
            if (k >= G->nc[a]) k = G->nc[a] - 1;
            c[a] = k;
        }
        size_t id = ((size_t)c[0] * G->nc[1] + c[1]) * G->nc[2] + c[2];
        G->next[i] = G->head[id];
        G->head[id] = i;
    }
    G->use = 1;
    return ORC_OK;
}

static void grid_free(orc_grid *G)
{
    free(G->head); free(G->next);
    memset(G, 0, sizeof(*G));
}

static int query_grid(const orc_sys *S, const orc_grid *G, int i, double rc, orc_list *out)
{
    const double *xi = S->pos + 3 * i;
    int c[3];
    for (int a = 0; a < 3; ++a) {
        double x = xi[a];
        if (S->pbc[a]) x -= S->box[a] * floor(x / S->box[a]);
        int k = (int)floor((x - G->lo[a]) / G->lc[a]);
        if (k < 0) k = 0;
        if (k >= G->nc[a]) k = G->nc[a] - 1;
        c[a] = k;
    }
    double rc2 = rc * rc;
    for (int o0 = -1; o0 <= 1; ++o0)
        for (int o1 = -1; o1 <= 1; ++o1)
            for (int o2 = -1; o2 <= 1; ++o2) {
                int cc[3] = {c[0] + o0, c[1] + o1, c[2] + o2}, skip = 0;
                for (int a = 0; a < 3; ++a) {
                    if (S->pbc[a]) cc[a] = (cc[a] + G->nc[a]) % G->nc[a];
                    else if (cc[a] < 0 || cc[a] >= G->nc[a]) skip = 1;
                }
                if (skip) continue;
                size_t id = ((size_t)cc[0] * G->nc[1] + cc[1]) * G->nc[2] + cc[2];
                for (int j = G->head[id]; j >= 0; j = G->next[j]) {
                    if (j == i) continue;
                    double d[3];
                    for (int a = 0; a < 3; ++a) {
                        d[a] = S->pos[3 * j + a] - xi[a];
                        if (S->pbc[a]) d[a] -= S->box[a] * floor(d[a] / S->box[a] + 0.5);
                    }
                    if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2 &&
                        list_push(out, j, sys_type(S, j), d))
                        return ORC_ERR_MEM;
                }
            }
    return ORC_OK;
}

static int query(const orc_sys *S, const orc_grid *G, int i, double rc, orc_list *out)
{
    return (G && G->use) ? query_grid(S, G, i, rc, out) : query_brute(S, i, rc, out);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Neighbour counts of every atom within rc (for tests: brute vs grid, shell
 * counts).  mode 0 = brute force, 1 = cell grid (falls back to brute force
 * when the box is too small). Also returns the sorted distances if dist is
 * given (row i holds counts[i] entries, at most maxn). */
int orc_neighbor_counts(int N, const double *pos, const double *box, const int *pbc,
                        double rc, int mode, int *counts, int maxn, double *dist)
{
    orc_sys S = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, NULL, 0, {0}, {0}};
    if (!sys_cell(&S, box)) return ORC_ERR_ARG;
    orc_grid G;
    memset(&G, 0, sizeof(G));
    if (mode == 1 && grid_build(&S, rc, &G)) return ORC_ERR_MEM;
    int err = ORC_OK;
    for (int i = 0; i < N && !err; ++i) {
        orc_list L;
        memset(&L, 0, sizeof(L));
        err = query(&S, &G, i, rc, &L);
        counts[i] = L.n;
        if (dist && !err) {
            /* the distances in ascending order, at most maxn of them */
            double *r = (double *)malloc(sizeof(double) * (size_t)(L.n + 1));
            for (int s = 0; s < L.n; ++s)
                r[s] = sqrt(L.d[3 * s] * L.d[3 * s] + L.d[3 * s + 1] * L.d[3 * s + 1] +
                            L.d[3 * s + 2] * L.d[3 * s + 2]);
            qsort(r, (size_t)L.n, sizeof(double), cmp_double);
            double *row = dist + (size_t)i * maxn;
            for (int s = 0; s < L.n && s < maxn; ++s) row[s] = r[s];
            free(r);
        }
        list_free(&L);
    }
    grid_free(&G);
    return err;
}

/* ---------------------------------------------------------------------------
 * Energy, forces, virial
 * ------------------------------------------------------------------------- */

typedef struct {
    orc_list R, A, Z;   /* radial (rcR), angular (rcA) and ZBL (zr2) lists */
    double U;           /* U_i (NEP + half of the ZBL pair terms) */
    double cond[4];     /* conditioning of the site (see site_nep) */
} orc_atom;

/* Lists and site gradients of atom i. */
static int atom_eval(const orc_model *m, const orc_sys *S, const orc_grid *G, int i,
                     orc_atom *at, double *q)
{
    memset(at, 0, sizeof(*at));
    int err = query(S, G, i, m->rcR, &at->R);
    if (!err) err = query(S, G, i, m->rcA, &at->A);
    if (!err) err = query(S, G, i, m->zr2, &at->Z);
    if (err) return err;
    at->R.g = (double *)malloc(sizeof(double) * 3 * (size_t)(at->R.n + 1));
    at->A.g = (double *)malloc(sizeof(double) * 3 * (size_t)(at->A.n + 1));
    at->Z.g = (double *)malloc(sizeof(double) * 3 * (size_t)(at->Z.n + 1));
    if (!at->R.g || !at->A.g || !at->Z.g) return ORC_ERR_MEM;
    const int ti = sys_type(S, i);
    at->U = site_nep(m, ti, at->R.n, at->R.d, at->R.t, at->A.n, at->A.d, at->A.t, q, at->R.g,
                     at->A.g, at->cond);
    for (int s = 0; s < at->Z.n; ++s) {
        const double *d = at->Z.d + 3 * s;
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double U, dU;
        orc_zbl(r, m->Z[ti], m->Z[at->Z.t[s]], m->zr1, m->zr2, &U, &dU);
        at->U += 0.5 * U;                                     /* Eq. 1 */
        for (int a = 0; a < 3; ++a) at->Z.g[3 * s + a] = 0.5 * dU * d[a] / r;
    }
    return ORC_OK;
}

static void atom_free(orc_atom *at)
{
    list_free(&at->R); list_free(&at->A); list_free(&at->Z);
}

static void accumulate(const orc_list *L, int i, double *F, double *W)
{
    for (int s = 0; s < L->n; ++s) {
        const double *g = L->g + 3 * s, *d = L->d + 3 * s;
        int j = L->j[s];
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += g[a];
            F[3 * j + a] -= g[a];
            for (int b = 0; b < 3; ++b) W[3 * a + b] -= g[a] * d[b];
        }
    }
}

static int efv(const orc_model *m, const orc_sys *S, int use_grid, double *E, double *F,
               double *W, double *Usite, double *qall)
{
    orc_grid G;
    memset(&G, 0, sizeof(G));
    if (use_grid && grid_build(S, m->rcR, &G)) return ORC_ERR_MEM;
    int N = S->N;
    orc_atom *atoms = (orc_atom *)calloc((size_t)(N > 0 ? N : 1), sizeof(orc_atom));
    if (!atoms) { grid_free(&G); return ORC_ERR_MEM; }
    int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < N; ++i) {
        int e = atom_eval(m, S, &G, i, &atoms[i], qall ? qall + (size_t)i * m->D : NULL);
        if (e) {
#pragma omp critical
            err = e;
        }
    }
    double Et = 0.0, Wt[9] = {0};
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)N);
    for (int i = 0; i < N && !err; ++i) {
        Et += atoms[i].U;
        if (Usite) Usite[i] = atoms[i].U;
        if (F) {
            accumulate(&atoms[i].R, i, F, Wt);
            accumulate(&atoms[i].A, i, F, Wt);
            accumulate(&atoms[i].Z, i, F, Wt);
        }
    }
    for (int i = 0; i < N; ++i) atom_free(&atoms[i]);
    free(atoms);
    grid_free(&G);
    if (E) *E = Et;
    if (W) memcpy(W, Wt, sizeof(Wt));
    return err;
}

/* Total energy E (eV), forces F (N,3) (eV/A), virial W (3x3 row-major, eV) and
 * site energies U (N) of a system.  use_grid = 0 forces brute-force
 * neighbours.  Any output pointer may be NULL. */
int orc_energy_forces_virial(const int *ihp, const double *dhp, const double *params,
                             const double *scaler, int N, const double *pos,
                             const int *types, const double *box, const int *pbc,
                             int use_grid, double *E, double *F, double *W, double *U)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler) || N < 0) return ORC_ERR_ARG;
    orc_sys S = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, types, 0, {0}, {0}};
    if (!sys_cell(&S, box)) return ORC_ERR_ARG;
    if (!types_valid(&S, m.T)) return ORC_ERR_ARG;
    return efv(&m, &S, use_grid, E, F, W, U, NULL);
}

#define NSCALE 5   /* rounding-error scales per atom (orc_force_scales) */

/* Magnitude of a pair gradient vector. */
static double norm3(const double *g)
{
    return sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

/* Rounding-error scales of every atom (test support; N x NSCALE):
 *   [0] S: sum of |g| over the NEP pair terms that enter F_i (its own lists'
 *       terms and its neighbours' terms pointing at it);
 *   [1] Z: the same over the ZBL pair terms;
 *   [2] W: the NEP pair terms' magnitudes weighted by the conditioning of
 *       the site they come from, sum |g| sqrt(M_k) max_mu sum_nu
 *       |w0_{mu nu} s_nu q_{k nu}| (k: the atom whose site energy the term
 *       differentiates, M_k its radial neighbours): the scale of the error
 *       that rounding of the descriptor sums passes through the adjoint;
 *   [3] sqrt(M_i) sum_mu |w1_mu (1 - t_mu^2)| sum_nu |w0 s q_i|: the scale of
 *       the site energy's response to that rounding;
 *   [4] sum_mu |w1_mu t_mu| + |b1|: the magnitude of U_i^NEP's terms. */
int orc_force_scales(const int *ihp, const double *dhp, const double *params,
                     const double *scaler, int N, const double *pos, const int *types,
                     const double *box, const int *pbc, int use_grid, double *sc)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler) || N < 0) return ORC_ERR_ARG;
    orc_sys Sy = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, types, 0, {0}, {0}};
    if (!sys_cell(&Sy, box)) return ORC_ERR_ARG;
    if (!types_valid(&Sy, m.T)) return ORC_ERR_ARG;
    orc_grid G;
    memset(&G, 0, sizeof(G));
    if (use_grid && grid_build(&Sy, m.rcR, &G)) return ORC_ERR_MEM;
    orc_atom *atoms = (orc_atom *)calloc((size_t)(N > 0 ? N : 1), sizeof(orc_atom));
    if (!atoms) { grid_free(&G); return ORC_ERR_MEM; }
    int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < N; ++i) {
        int e = atom_eval(&m, &Sy, &G, i, &atoms[i], NULL);
        if (e) {
#pragma omp critical
            err = e;
        }
    }
    memset(sc, 0, sizeof(double) * NSCALE * (size_t)N);
    for (int i = 0; i < N && !err; ++i) {
        const double ki = sqrt(atoms[i].cond[0]) * atoms[i].cond[1];
        double *oi = sc + (size_t)NSCALE * i;
        oi[3] = sqrt(atoms[i].cond[0]) * atoms[i].cond[2];
        oi[4] = atoms[i].cond[3];
        const orc_list *Ls[3] = {&atoms[i].R, &atoms[i].A, &atoms[i].Z};
        for (int w = 0; w < 3; ++w) {
            const int col = w < 2 ? 0 : 1;
            for (int s = 0; s < Ls[w]->n; ++s) {
                const int j = Ls[w]->j[s];
                if (j == i) continue;   /* a self-image term cancels in F_i */
                const double v = norm3(Ls[w]->g + 3 * s);
                oi[col] += v;
                sc[(size_t)NSCALE * j + col] += v;
                if (col == 0) {   /* a term of atom i's site energy */
                    oi[2] += v * ki;
                    sc[(size_t)NSCALE * j + 2] += v * ki;
                }
            }
        }
    }
    for (int i = 0; i < N; ++i) atom_free(&atoms[i]);
    free(atoms);
    grid_free(&G);
    return err;
}

/* Unscaled descriptors q (N, D) of every atom. */
int orc_descriptors(const int *ihp, const double *dhp, const double *params,
                    const double *scaler, int N, const double *pos, const int *types,
                    const double *box, const int *pbc, int use_grid, double *q)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler) || N < 0) return ORC_ERR_ARG;
    orc_sys S = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, types, 0, {0}, {0}};
    if (!sys_cell(&S, box)) return ORC_ERR_ARG;
    if (!types_valid(&S, m.T)) return ORC_ERR_ARG;
    return efv(&m, &S, use_grid, NULL, NULL, NULL, NULL, q);
}

/* Forces and site energies of a subset of atoms idx[nidx] only (for sampled
 * comparisons on large systems):
 *   F_a = sum_{s in lists(a), j_s != a} g_{a,s} - sum_{k != a} sum_{t: j_t = a} g_{k,t}
 * where k runs over the distinct atoms in the radial neighbourhood of a.
 * Optionally (sc not NULL, nidx x NSCALE) the scales of each listed atom's
 * force and site energy for rounding-error bounds (see scales_of). */
static int forces_subset(const int *ihp, const double *dhp, const double *params,
                         const double *scaler, int N, const double *pos, const int *types,
                         const double *box, const int *pbc, int nidx, const int64_t *idx,
                         double *F, double *U, double *sc)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler) || N < 0) return ORC_ERR_ARG;
    orc_sys Sy = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, types, 0, {0}, {0}};
    if (!sys_cell(&Sy, box)) return ORC_ERR_ARG;
    if (!types_valid(&Sy, m.T)) return ORC_ERR_ARG;
    orc_grid G;
    memset(&G, 0, sizeof(G));
    if (grid_build(&Sy, m.rcR, &G)) return ORC_ERR_MEM;
    int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nidx; ++t) {
        int a = (int)idx[t];
        double f[3] = {0, 0, 0}, sn = 0.0, sz = 0.0, sw = 0.0;
        orc_atom at;
        int e = atom_eval(&m, &Sy, &G, a, &at, NULL);
        if (!e) {
            U[t] = at.U;
            const double ka = sqrt(at.cond[0]) * at.cond[1];
            const orc_list *Ls[3] = {&at.R, &at.A, &at.Z};
            for (int w = 0; w < 3; ++w)
                for (int s = 0; s < Ls[w]->n; ++s)
                    if (Ls[w]->j[s] != a) {
                        for (int c = 0; c < 3; ++c) f[c] += Ls[w]->g[3 * s + c];
                        const double v = norm3(Ls[w]->g + 3 * s);
                        if (w < 2) { sn += v; sw += v * ka; }
                        else sz += v;
                    }
            /* distinct neighbours k != a */
            int nk = 0;
            int *ks = (int *)malloc(sizeof(int) * (size_t)(at.R.n + 1));
            for (int s = 0; s < at.R.n; ++s) {
                int k = at.R.j[s], dup = 0;
                if (k == a) continue;
                for (int u = 0; u < nk; ++u) if (ks[u] == k) { dup = 1; break; }
                if (!dup) ks[nk++] = k;
            }
            for (int u = 0; u < nk && !e; ++u) {
                orc_atom bk;
                e = atom_eval(&m, &Sy, &G, ks[u], &bk, NULL);
                if (!e) {
                    const double kk = sqrt(bk.cond[0]) * bk.cond[1];
                    const orc_list *Lk[3] = {&bk.R, &bk.A, &bk.Z};
                    for (int w = 0; w < 3; ++w)
                        for (int s = 0; s < Lk[w]->n; ++s)
                            if (Lk[w]->j[s] == a) {
                                for (int c = 0; c < 3; ++c) f[c] -= Lk[w]->g[3 * s + c];
                                const double v = norm3(Lk[w]->g + 3 * s);
                                if (w < 2) { sn += v; sw += v * kk; }
                                else sz += v;
                            }
                }
                atom_free(&bk);
            }
            free(ks);
        }
        atom_free(&at);
        for (int c = 0; c < 3; ++c) F[3 * t + c] = f[c];
        if (sc) {
            double *o = sc + (size_t)NSCALE * t;
            o[0] = sn;
            o[1] = sz;
            o[2] = sw;
            o[3] = sqrt(at.cond[0]) * at.cond[2];
            o[4] = at.cond[3];
        }
        if (e) {
#pragma omp critical
            err = e;
        }
    }
    grid_free(&G);
    return err;
}

int orc_forces_subset(const int *ihp, const double *dhp, const double *params,
                      const double *scaler, int N, const double *pos, const int *types,
                      const double *box, const int *pbc, int nidx, const int64_t *idx,
                      double *F, double *U)
{
    return forces_subset(ihp, dhp, params, scaler, N, pos, types, box, pbc, nidx, idx, F, U,
                         NULL);
}

/* orc_forces_subset plus the rounding-error scales (nidx x NSCALE, see
 * scales_of) of each listed atom. */
int orc_forces_subset_scales(const int *ihp, const double *dhp, const double *params,
                             const double *scaler, int N, const double *pos, const int *types,
                             const double *box, const int *pbc, int nidx, const int64_t *idx,
                             double *F, double *U, double *sc)
{
    return forces_subset(ihp, dhp, params, scaler, N, pos, types, box, pbc, nidx, idx, F, U, sc);
}

/* ---------------------------------------------------------------------------
 * Velocity-Verlet NVE (Sec. II.B; variable time step of Sec. II.B)
 * ------------------------------------------------------------------------- */

/* Advances pos/vel (N,3) by nsteps.  dt = min(dt_max, d_max / max_i |v_i|)
 * before each step when d_max > 0, else dt = dt_max (fs).  Periodic
 * coordinates are wrapped into [0, L).  thermo (nsteps x 4, may be NULL)
 * receives t, dt, potential and kinetic energy after each step.  F (N,3) holds
 * the forces at the initial positions on entry when forces_valid != 0, and
 * the final forces on return.  mass[t] is the mass (amu) of species t. */
int orc_md(const int *ihp, const double *dhp, const double *params, const double *scaler,
           int N, double *pos, double *vel, double *F, int forces_valid, const int *types,
           const double *box, const int *pbc, const double *mass, double dt_max,
           double d_max, int nsteps, int use_grid, double *thermo)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler) || N < 0) return ORC_ERR_ARG;
    for (int t = 0; t < m.T; ++t)
        if (!(mass[t] > 0)) return ORC_ERR_ARG;
    orc_sys S = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, types, 0, {0}, {0}};
    if (!sys_cell(&S, box)) return ORC_ERR_ARG;
    if (!types_valid(&S, m.T)) return ORC_ERR_ARG;
    double E, W[9];
    int err = ORC_OK;
    if (!forces_valid) err = efv(&m, &S, use_grid, &E, F, W, NULL, NULL);
    double t = 0.0;
    for (int step = 0; step < nsteps && !err; ++step) {
        double dt = dt_max;
        if (d_max > 0) {
            double vmax = 0.0;
            for (int i = 0; i < N; ++i) {
                double v = sqrt(vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                                vel[3 * i + 2] * vel[3 * i + 2]);
                if (v > vmax) vmax = v;
            }
            if (vmax > 0 && d_max / vmax < dt) dt = d_max / vmax;
        }
        for (int i = 0; i < 3 * N; ++i) {
            const double acc = ORC_EV_AMU / mass[sys_type(&S, i / 3)];
            vel[i] += 0.5 * dt * F[i] * acc;
            pos[i] += dt * vel[i];
        }
        for (int i = 0; i < N; ++i) {
            if (S.tric) { wrap_tric(&S, pos + 3 * i); continue; }
            for (int a = 0; a < 3; ++a)
                if (pbc[a]) pos[3 * i + a] -= S.box[a] * floor(pos[3 * i + a] / S.box[a]);
        }
        err = efv(&m, &S, use_grid, &E, F, W, NULL, NULL);
        double ke = 0.0;
        for (int i = 0; i < 3 * N; ++i) {
            const double mi = mass[sys_type(&S, i / 3)];
            vel[i] += 0.5 * dt * F[i] * (ORC_EV_AMU / mi);
            ke += 0.5 * mi * vel[i] * vel[i] / ORC_EV_AMU;
        }
        t += dt;
        if (thermo) {
            thermo[4 * step + 0] = t;
            thermo[4 * step + 1] = dt;
            thermo[4 * step + 2] = E;
            thermo[4 * step + 3] = ke;
        }
    }
    return err;
}

/* ---------------------------------------------------------------------------
 * Cascade protocol pieces (Sec. II.B): a Nose-Hoover chain thermostat on a
 * group of atoms (Martyna, Klein and Tuckerman 1992) and a Berendsen
 * barostat for the NPT equilibration at a target pressure.
 *
 * One step of length dt (Trotter splitting, as in Martyna, Tuckerman, Tobias
 * and Klein 1996, one Suzuki-Yoshida weight):
 *   NHC(dt/2) ; v += dt/2 F/m ; x += dt v ; F(x) ; v += dt/2 F/m ; NHC(dt/2) ;
 *   then, with a barostat, x_a *= mu_a and L_a *= mu_a for every periodic a,
 *   mu_a = [1 - beta (dt / tau_p) (p0 - P_aa)]^(1/3),
 *   P_aa = (sum_i m_i v_ia^2 + W_aa) / V   (W: the virial of the new positions).
 * NHC(d) for the group g (N_f = 3 N_g, Q_1 = N_f kT tau^2, Q_j = kT tau^2,
 * G_1 = (2 K_g - N_f kT) / Q_1, G_j = (Q_{j-1} v_{j-1}^2 - kT) / Q_j):
 *   v_M += d/2 G_M;
 *   for j = M-1..1: v_j *= e^{-d/4 v_{j+1}}; v_j += d/2 G_j; v_j *= e^{-d/4 v_{j+1}}
 *   s = e^{-d v_1}: group velocities *= s, K_g *= s^2;  xi_j += d v_j
 *   for j = 1..M-1: v_j *= e^{-d/4 v_{j+1}}; v_j += d/2 G_j; v_j *= e^{-d/4 v_{j+1}}
 *   v_M += d/2 G_M
 * (each G evaluated with the current values).  The thermostat energy
 * sum_j Q_j v_j^2 / 2 + N_f kT xi_1 + kT sum_{j>1} xi_j makes
 * PE + KE + E_NHC a constant of the motion.
 * ------------------------------------------------------------------------- */

#define ORC_KB 8.617333262e-5   /* eV/K */
#define ORC_MAXCHAIN 8

typedef struct {
    int M;
    double kT, Nf, Q[ORC_MAXCHAIN], v[ORC_MAXCHAIN], xi[ORC_MAXCHAIN];
} orc_nhc;

static double nhc_G(const orc_nhc *c, int j, double Kg)
{
    if (j == 0) return (2.0 * Kg - c->Nf * c->kT) / c->Q[0];
    return (c->Q[j - 1] * c->v[j - 1] * c->v[j - 1] - c->kT) / c->Q[j];
}

static void nhc_sub(orc_nhc *c, int j, double d, double Kg)
{
    if (j + 1 < c->M) c->v[j] *= exp(-0.25 * d * c->v[j + 1]);
    c->v[j] += 0.5 * d * nhc_G(c, j, Kg);
    if (j + 1 < c->M) c->v[j] *= exp(-0.25 * d * c->v[j + 1]);
}

/* One NHC(d) sweep; returns the velocity scale of the group. */
static double nhc_half(orc_nhc *c, double d, double Kg)
{
    const int M = c->M;
    for (int j = M - 1; j >= 0; --j) nhc_sub(c, j, d, Kg);
    const double s = exp(-d * c->v[0]);
    Kg *= s * s;
    for (int j = 0; j < M; ++j) c->xi[j] += d * c->v[j];
    for (int j = 0; j < M; ++j) nhc_sub(c, j, d, Kg);
    return s;
}

static double nhc_energy(const orc_nhc *c)
{
    double e = 0.0;
    for (int j = 0; j < c->M; ++j) e += 0.5 * c->Q[j] * c->v[j] * c->v[j];
    e += c->Nf * c->kT * c->xi[0];
    for (int j = 1; j < c->M; ++j) e += c->kT * c->xi[j];
    return e;
}

static double group_ke(int N, const double *vel, const int *types, const double *mass,
                       const unsigned char *group)
{
    double k = 0.0;
    for (int i = 0; i < N; ++i) {
        if (group && !group[i]) continue;
        const double mi = mass[types ? types[i] : 0];
        for (int a = 0; a < 3; ++a) k += 0.5 * mi * vel[3 * i + a] * vel[3 * i + a] / ORC_EV_AMU;
    }
    return k;
}

/* Velocity Verlet with the optional thermostat and barostat above.
 * ext = {T (K), tau (fs), chain length, p0 (eV/A^3), tau_p (fs), beta (A^3/eV)};
 * the thermostat is on when thermostat != 0 (group: N flags, NULL = all
 * atoms), the barostat when tau_p > 0 (orthorhombic cells only).  box (H,
 * 9 doubles) is updated in place.
 * thermo (nsteps x 8): t, dt, PE, KE, E_NHC, Lx, Ly, Lz after each step. */
int orc_md_ext(const int *ihp, const double *dhp, const double *params, const double *scaler,
               int N, double *pos, double *vel, double *F, int forces_valid, const int *types,
               double *box, const int *pbc, const double *mass, double dt_max, double d_max,
               int nsteps, int use_grid, int thermostat, const unsigned char *group,
               const double *ext, double *thermo)
{
    orc_model m;
    if (model_init(&m, ihp, dhp, params, scaler) || N < 0) return ORC_ERR_ARG;
    for (int t = 0; t < m.T; ++t)
        if (!(mass[t] > 0)) return ORC_ERR_ARG;
    orc_sys S = {N, pos, {0, 0, 0}, {pbc[0], pbc[1], pbc[2]}, types, 0, {0}, {0}};
    if (!sys_cell(&S, box)) return ORC_ERR_ARG;
    if (!types_valid(&S, m.T)) return ORC_ERR_ARG;
    orc_nhc c;
    memset(&c, 0, sizeof(c));
    if (thermostat) {
        c.M = (int)ext[2];
        if (c.M < 1 || c.M > ORC_MAXCHAIN || !(ext[0] > 0) || !(ext[1] > 0)) return ORC_ERR_ARG;
        int ng = 0;
        for (int i = 0; i < N; ++i) ng += group ? (group[i] != 0) : 1;
        c.kT = ORC_KB * ext[0];
        c.Nf = 3.0 * ng;
        c.Q[0] = (c.Nf > 0 ? c.Nf : 1.0) * c.kT * ext[1] * ext[1];
        for (int j = 1; j < c.M; ++j) c.Q[j] = c.kT * ext[1] * ext[1];
    }
    const int baro = ext && ext[4] > 0;
    if (baro && S.tric) return ORC_ERR_ARG;          /* the barostat scales an orthorhombic box */
    double E, W[9];
    int err = ORC_OK;
    if (!forces_valid) err = efv(&m, &S, use_grid, &E, F, W, NULL, NULL);
    double t = 0.0;
    for (int step = 0; step < nsteps && !err; ++step) {
        double dt = dt_max;
        if (d_max > 0) {
            double vmax = 0.0;
            for (int i = 0; i < N; ++i) {
                double v = sqrt(vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                                vel[3 * i + 2] * vel[3 * i + 2]);
                if (v > vmax) vmax = v;
            }
            if (vmax > 0 && d_max / vmax < dt) dt = d_max / vmax;
        }
        if (thermostat) {
            const double sc = nhc_half(&c, 0.5 * dt, group_ke(N, vel, types, mass, group));
            for (int i = 0; i < N; ++i)
                if (!group || group[i])
                    for (int a = 0; a < 3; ++a) vel[3 * i + a] *= sc;
        }
        for (int i = 0; i < 3 * N; ++i) {
            const double acc = ORC_EV_AMU / mass[sys_type(&S, i / 3)];
            vel[i] += 0.5 * dt * F[i] * acc;
            pos[i] += dt * vel[i];
        }
        for (int i = 0; i < N; ++i) {
            if (S.tric) { wrap_tric(&S, pos + 3 * i); continue; }
            for (int a = 0; a < 3; ++a)
                if (pbc[a]) pos[3 * i + a] -= S.box[a] * floor(pos[3 * i + a] / S.box[a]);
        }
        err = efv(&m, &S, use_grid, &E, F, W, NULL, NULL);
        for (int i = 0; i < 3 * N; ++i)
            vel[i] += 0.5 * dt * F[i] * (ORC_EV_AMU / mass[sys_type(&S, i / 3)]);
        if (thermostat) {
            const double sc = nhc_half(&c, 0.5 * dt, group_ke(N, vel, types, mass, group));
            for (int i = 0; i < N; ++i)
                if (!group || group[i])
                    for (int a = 0; a < 3; ++a) vel[3 * i + a] *= sc;
        }
        double ke = 0.0, kab[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < N; ++i) {
            const double mi = mass[sys_type(&S, i)];
            for (int a = 0; a < 3; ++a) {
                ke += 0.5 * mi * vel[3 * i + a] * vel[3 * i + a] / ORC_EV_AMU;
                kab[a] += mi * vel[3 * i + a] * vel[3 * i + a] / ORC_EV_AMU;
            }
        }
        t += dt;
        if (baro && !err) {
            const double V = S.box[0] * S.box[1] * S.box[2];
            for (int a = 0; a < 3; ++a) {
                if (!pbc[a]) continue;
                const double P = (kab[a] + W[4 * a]) / V;
                const double mu = cbrt(1.0 - ext[5] * (dt / ext[4]) * (ext[3] - P));
                for (int i = 0; i < N; ++i) pos[3 * i + a] *= mu;
                S.box[a] *= mu;
                S.h[4 * a] = S.box[a];
                S.hinv[4 * a] = 1.0 / S.box[a];
                box[4 * a] = S.box[a];
            }
        }
        if (thermo) {
            double *o = thermo + 8 * (size_t)step;
            o[0] = t; o[1] = dt; o[2] = E; o[3] = ke;
            o[4] = thermostat ? nhc_energy(&c) : 0.0;
            o[5] = S.box[0]; o[6] = S.box[1]; o[7] = S.box[2];
        }
    }
    return err;
}
