/*
 * Plain C versions of the oracle's two expensive loops (test infrastructure
 * only; see oracle/__init__.py).  They compute exactly what
 * oracle.integrals.pair_blocks and oracle.pfft.Pfft.grid_blocks compute, in
 * FP64, one triangle pair at a time, and are pinned against those numpy
 * versions by tests/test_oracle_integrals.py::test_native_potentials_match
 * and tests/test_oracle_pfft.py::test_native_grid_blocks_match.
 *
 * orc_pair_blocks  : Eq. (Zb) inductive 3x3 block of a triangle pair, inner
 *                    integral over the second triangle in closed form (sum over
 *                    its edges of logarithms and arctangents), outer rule on
 *                    the first triangle.
 * orc_grid_blocks  : the pFFT grid product (I H B) of Sec. IV-B restricted to a
 *                    triangle pair, written as the plain double sum over the
 *                    two stencils of every pair of sample points.
 */
#include <math.h>
#include <stdint.h>

static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* K0 = int_T 1/|r-r'| dS', K1 = int_T (rho'-rho)/|r-r'| dS' over triangle v[0..2]. */
static void potentials(const double *r, const double *v, double *K0, double *K1) {
    double e1[3], e2[3], n[3], d[3], rho[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, n);
    double nn = norm3(n);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    sub3(r, v, d);
    double h = dot3(d, n), ah = fabs(h);
    rho[0] = r[0] - h * n[0]; rho[1] = r[1] - h * n[1]; rho[2] = r[2] - h * n[2];
    double k0 = 0.0, k1[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const double *pm = v + 3 * i, *pp = v + 3 * ((i + 1) % 3);
        double L[3], lt[3], u[3], a[3], b[3], ra[3], rb[3];
        sub3(pp, pm, L);
        double ll = norm3(L);
        lt[0] = L[0] / ll; lt[1] = L[1] / ll; lt[2] = L[2] / ll;
        cross3(lt, n, u);
        sub3(pp, rho, a);
        sub3(pm, rho, b);
        double lp = dot3(a, lt), lm = dot3(b, lt), P0 = dot3(b, u);
        double R0s = P0 * P0 + h * h;
        sub3(r, pp, ra);
        sub3(r, pm, rb);
        double Rp = norm3(ra), Rm = norm3(rb);
        double f = 0.0;
        if (R0s > 0.0) {
            double num = lp >= 0.0 ? Rp + lp : R0s / (Rp - lp);
            double den = lm >= 0.0 ? Rm + lm : R0s / (Rm - lm);
            f = log(num / den);
        }
        double beta = atan2(P0 * lp, R0s + ah * Rp) - atan2(P0 * lm, R0s + ah * Rm);
        k0 += P0 * f - ah * beta;
        double s = 0.5 * (R0s * f + lp * Rp - lm * Rm);
        k1[0] += s * u[0]; k1[1] += s * u[1]; k1[2] += s * u[2];
    }
    *K0 = k0;
    K1[0] = k1[0]; K1[1] = k1[1]; K1[2] = k1[2];
}

/*
 * pT, pS: [m][3][3] vertices (outer, inner); aT, aS: [m] areas;
 * bary: [Q][3], w: [Q] outer rule; out: [m][3][3].
 * out[k][l] = sum_q w_q A_T (r_q - v_k).(K1 + (rho_q - v'_l) K0) / (4 A_T A_S)
 */
void orc_pair_blocks(int64_t m, const double *pT, const double *aT, const double *pS,
                     const double *aS, int64_t Q, const double *bary, const double *w,
                     double *out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < m; ++t) {
        const double *vT = pT + 9 * t, *vS = pS + 9 * t;
        double n[3], e1[3], e2[3];
        sub3(vS + 3, vS, e1);
        sub3(vS + 6, vS, e2);
        cross3(e1, e2, n);
        double nn = norm3(n);
        n[0] /= nn; n[1] /= nn; n[2] /= nn;
        double acc[9] = {0};
        for (int64_t q = 0; q < Q; ++q) {
            double r[3], K0, K1[3], d[3], rho[3];
            for (int c = 0; c < 3; ++c)
                r[c] = bary[3 * q] * vT[c] + bary[3 * q + 1] * vT[3 + c] + bary[3 * q + 2] * vT[6 + c];
            potentials(r, vS, &K0, K1);
            sub3(r, vS, d);
            double h = dot3(d, n);
            for (int c = 0; c < 3; ++c) rho[c] = r[c] - h * n[c];
            for (int k = 0; k < 3; ++k) {
                double o[3];
                sub3(r, vT + 3 * k, o);
                for (int l = 0; l < 3; ++l) {
                    double in[3];
                    for (int c = 0; c < 3; ++c) in[c] = K1[c] + (rho[c] - vS[3 * l + c]) * K0;
                    acc[3 * k + l] += w[q] * dot3(o, in);
                }
            }
        }
        double s = aT[t] / (4.0 * aT[t] * aS[t]);
        for (int i = 0; i < 9; ++i) out[9 * t + i] = acc[i] * s;
    }
}

/*
 * Grid product (I H B) for triangle pairs (ti[p], tj[p]).
 * start: [nt][Q][3] stencil start nodes; lw: [3][nt][Q][O] Lagrange weights;
 * mom: [nt][Q][3][3] point moments (w_q/2)(r_q - v_k); Hpad: padded kernel table
 * [Mx][My][Mz] indexed by offset modulo M; out: [npairs][3][3].
 */
void orc_grid_blocks(int64_t npairs, const int64_t *ti, const int64_t *tj, int64_t nt, int64_t Q,
                     int64_t O, const int64_t *start, const double *lw, const double *mom,
                     const double *Hpad, int64_t Mx, int64_t My, int64_t Mz, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t a = ti[p], b = tj[p];
        double acc[9] = {0};
        for (int64_t q = 0; q < Q; ++q) {
            const int64_t *sa = start + 3 * (a * Q + q);
            const double *wxa = lw + (0 * nt * Q + a * Q + q) * O;
            const double *wya = lw + (1 * nt * Q + a * Q + q) * O;
            const double *wza = lw + (2 * nt * Q + a * Q + q) * O;
            for (int64_t r = 0; r < Q; ++r) {
                const int64_t *sb = start + 3 * (b * Q + r);
                const double *wxb = lw + (0 * nt * Q + b * Q + r) * O;
                const double *wyb = lw + (1 * nt * Q + b * Q + r) * O;
                const double *wzb = lw + (2 * nt * Q + b * Q + r) * O;
                double G = 0.0;
                for (int64_t i = 0; i < O; ++i)
                    for (int64_t j = 0; j < O; ++j)
                        for (int64_t k = 0; k < O; ++k) {
                            double la = wxa[i] * wya[j] * wza[k];
                            for (int64_t i2 = 0; i2 < O; ++i2)
                                for (int64_t j2 = 0; j2 < O; ++j2)
                                    for (int64_t k2 = 0; k2 < O; ++k2) {
                                        int64_t dx = (sa[0] + i) - (sb[0] + i2);
                                        int64_t dy = (sa[1] + j) - (sb[1] + j2);
                                        int64_t dz = (sa[2] + k) - (sb[2] + k2);
                                        dx = ((dx % Mx) + Mx) % Mx;
                                        dy = ((dy % My) + My) % My;
                                        dz = ((dz % Mz) + Mz) % Mz;
                                        double lb = wxb[i2] * wyb[j2] * wzb[k2];
                                        G += la * Hpad[(dx * My + dy) * Mz + dz] * lb;
                                    }
                        }
                const double *fa = mom + 9 * (a * Q + q);
                const double *fb = mom + 9 * (b * Q + r);
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l)
                        acc[3 * k + l] += dot3(fa + 3 * k, fb + 3 * l) * G;
            }
        }
        for (int i = 0; i < 9; ++i) out[9 * p + i] = acc[i];
    }
}
