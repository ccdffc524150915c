/*
 * FP64 CPU oracle for the particle mesh multipole method (PMMM,
 * K. Nitadori, "Particle mesh multipole method", arXiv:1409.5981).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a stand-alone shared
 * library that only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg load.  The GPU library never includes, links or calls it, and
 * it shares no code, header, table or constant generator with the GPU path.
 *
 * Everything here is written from the definitions in the paper, in plain
 * loops, in double precision, with no blocking or reordering beyond what the
 * definition states:
 *
 *   solid harmonics R, S ............ App. A.1 (spherical definitions with the
 *                                      associated Legendre function of App. A.1;
 *                                      conjugate relation for m < 0)
 *   P2M, M2M, M2P, M2L, L2L, L2P .... App. A.3, Eqs. P2M, M2M, M2P, M2L, L2L, L2P
 *   gradient from L_1 ............... App. A.4, Eq. phigrad
 *   cell convolution L_i = sum G M .. Sec. 2.1, Eq. pmmm, summed over all cell
 *                                      pairs (no FFT): the definition itself
 *   open-boundary Green function .... Sec. 2.1 (mask of the nearest cells) and
 *                                      App. C (displacements up to +-(n-1) cells)
 *   periodic Green function ......... App. B, Eqs. infsum and greenPBC (Ewald
 *                                      split with incomplete gamma functions)
 *   periodic corrections ............ App. B.3 (correction procedure)
 *   near field ...................... Sec. 2.1/2.2: pure Newtonian 1/r over the
 *                                      masked (2c+1)^3 cells
 *   direct O(N^2) sum, Ewald sum .... Sec. 4 and App. B.3, Eq. refewald
 *   two-level PMMM .................. Sec. 5 (hierarchical treatment) and
 *                                      Fig. refine: PMMM on a coarse mesh plus
 *                                      free-space M2L between the fine cells of
 *                                      each masked coarse block, cell pair by
 *                                      cell pair
 *
 * Where the paper is ambiguous or its printed formula is defective, the
 * readings taken here are: the Ewald self term with a minus sign, q_j in the
 * real-space Ewald term, (-i pi)^l with exp(+2 pi i k.r), the n = 0 image
 * left out of the self cell, only the image with |cell offset|_inf <= c
 * masked, the FP64 binning formula, the forward DFT with exp(-2 pi i), and
 * for the two-level method the same cutoff at both levels with the periodic
 * corrections taken at the coarse level.
 *
 * Complex harmonic arrays use the full index l*l + l + m, m in [-l, l], as
 * interleaved (re, im) doubles: (p+1)^2 complex numbers for order p.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_VERSION 5
#define LMAX_ORACLE 48

static inline int hidx(int l, int m) { return l * l + l + m; }

int orc_version(void) { return ORC_VERSION; }

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* ------------------------------------------------------------------------ */
/* Associated Legendre functions (App. A.1): P_l^m(cos t) including the       */
/* factor (-1)^m of the definition P_l^m = (-sin t)^m d^m/d(cos t)^m P_l.     */
/* Textbook three-term recurrence in x = cos t with s = sin t supplied        */
/* separately (so that points near the axis keep full precision).             */
/* out[hidx(l, m)] for 0 <= m <= l <= lmax; negative-m slots are untouched.   */
/* ------------------------------------------------------------------------ */
void orc_legendre(int lmax, double x, double s, double *out)
{
    for (int m = 0; m <= lmax; ++m) {
        /* P_m^m = (-1)^m (2m-1)!! s^m */
        double pmm = 1.0;
        for (int i = 1; i <= m; ++i) pmm *= -(double)(2 * i - 1) * s;
        out[hidx(m, m)] = pmm;
        if (m == lmax) break;
        double pm1 = x * (double)(2 * m + 1) * pmm; /* P_{m+1}^m */
        out[hidx(m + 1, m)] = pm1;
        double a = pmm, b = pm1;
        for (int l = m + 2; l <= lmax; ++l) {
            double c = (x * (double)(2 * l - 1) * b - (double)(l + m - 1) * a) / (double)(l - m);
            out[hidx(l, m)] = c;
            a = b;
            b = c;
        }
    }
}

/* Spherical coordinates of r: radius, cos(theta), sin(theta), phi. */
static void spherical(const double r[3], double *rad, double *ct, double *st, double *ph)
{
    double rho = hypot(r[0], r[1]);
    *rad = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (*rad > 0.0) {
        *ct = r[2] / *rad;
        *st = rho / *rad;
    } else {
        *ct = 1.0;
        *st = 0.0;
    }
    *ph = atan2(r[1], r[0]);
}

/* R_l^m(r) = r^l / (l+m)! P_l^m(cos t) e^{i m phi},  R_l^{-m} = (-1)^m conj(R_l^m).
 * (App. A.1.)  out: (p+1)^2 complex, full index. */
static void solid_R(int p, const double r[3], cplx *out)
{
    double rad, ct, st, ph;
    double P[(LMAX_ORACLE + 1) * (LMAX_ORACLE + 1)];
    spherical(r, &rad, &ct, &st, &ph);
    orc_legendre(p, ct, st, P);
    for (int l = 0; l <= p; ++l) {
        double rl = pow(rad, (double)l);
        if (l == 0) rl = 1.0;
        for (int m = 0; m <= l; ++m) {
            cplx e = cos(m * ph) + I * sin(m * ph);
            cplx v = rl / factorial(l + m) * P[hidx(l, m)] * e;
            out[hidx(l, m)] = v;
            if (m > 0) out[hidx(l, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
}

/* S_l^m(r) = (-1)^{l+m} (l-m)! / r^{l+1} P_l^m(cos t) e^{i m phi},
 * S_l^{-m} = (-1)^m conj(S_l^m).  (App. A.1.)  r must be nonzero. */
static void solid_S(int p, const double r[3], cplx *out)
{
    double rad, ct, st, ph;
    double P[(LMAX_ORACLE + 1) * (LMAX_ORACLE + 1)];
    spherical(r, &rad, &ct, &st, &ph);
    orc_legendre(p, ct, st, P);
    for (int l = 0; l <= p; ++l) {
        double inv = 1.0 / pow(rad, (double)(l + 1));
        for (int m = 0; m <= l; ++m) {
            cplx e = cos(m * ph) + I * sin(m * ph);
            double sg = ((l + m) & 1) ? -1.0 : 1.0;
            cplx v = sg * factorial(l - m) * inv * P[hidx(l, m)] * e;
            out[hidx(l, m)] = v;
            if (m > 0) out[hidx(l, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
}

void orc_solid_R(int p, const double *r, double *out) { solid_R(p, r, (cplx *)out); }
void orc_solid_S(int p, const double *r, double *out) { solid_S(p, r, (cplx *)out); }

/* ------------------------------------------------------------------------ */
/* Regularised incomplete gamma functions for half-integer a = l + 1/2,      */
/* as used by the Ewald split of App. B.1:                                   */
/*   Q(a, x) = Gamma(a, x) / Gamma(a),   P(a, x) = gamma(a, x) / Gamma(a).   */
/* Q(1/2, x) = erfc(sqrt x); Q(a+1, x) = Q(a, x) + x^a e^{-x} / Gamma(a+1).  */
/* P by its power series when x < a + 1 (where 1 - Q would cancel), else     */
/* as 1 - Q.                                                                 */
/* ------------------------------------------------------------------------ */
double orc_gammaQ_half(int l, double x)
{
    double q = erfc(sqrt(x));
    double a = 0.5;
    for (int k = 0; k < l; ++k) {
        q += exp(a * log(x) - x - lgamma(a + 1.0));
        a += 1.0;
    }
    if (x == 0.0) q = 1.0;
    return q;
}

double orc_gammaP_half(int l, double x)
{
    double a = l + 0.5;
    if (x == 0.0) return 0.0;
    if (x < a + 1.0) {
        /* P(a,x) = x^a e^{-x} / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k)) */
        double term = 1.0, sum = 1.0;
        for (int k = 1; k < 1000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (term < 1e-17 * sum) break;
        }
        return exp(a * log(x) - x - lgamma(a + 1.0)) * sum;
    }
    return 1.0 - orc_gammaQ_half(l, x);
}

/* ------------------------------------------------------------------------ */
/* Translations (App. A.3)                                                   */
/* ------------------------------------------------------------------------ */

/* P2M: M_l^m = sum_i q_i R_l^m(r_M - r_i). Accumulates into M. */
static void p2m(int p, int64_t n, const double *pos, const double *q, const double c[3], cplx *M)
{
    int np = (p + 1) * (p + 1);
    cplx *R = (cplx *)malloc(sizeof(cplx) * np);
    for (int64_t i = 0; i < n; ++i) {
        double d[3] = {c[0] - pos[3 * i], c[1] - pos[3 * i + 1], c[2] - pos[3 * i + 2]};
        solid_R(p, d, R);
        for (int k = 0; k < np; ++k) M[k] += q[i] * R[k];
    }
    free(R);
}

void orc_p2m(int p, int64_t n, const double *pos, const double *q, const double *center, double *M)
{
    p2m(p, n, pos, q, center, (cplx *)M);
}

/* M2M: M'_l^m = sum_{lam=0..l} sum_mu M_{l-lam}^{m-mu} R_lam^mu(r_M' - r_M). */
void orc_m2m(int p, const double *Min, const double *shift, double *Mout)
{
    const cplx *M = (const cplx *)Min;
    cplx *Mo = (cplx *)Mout;
    int np = (p + 1) * (p + 1);
    cplx *R = (cplx *)malloc(sizeof(cplx) * np);
    solid_R(p, shift, R);
    for (int l = 0; l <= p; ++l)
        for (int m = -l; m <= l; ++m) {
            cplx acc = 0;
            for (int lam = 0; lam <= l; ++lam)
                for (int mu = -lam; mu <= lam; ++mu) {
                    int ls = l - lam, ms = m - mu;
                    if (ms < -ls || ms > ls) continue;
                    acc += M[hidx(ls, ms)] * R[hidx(lam, mu)];
                }
            Mo[hidx(l, m)] = acc;
        }
    free(R);
}

/* M2P: Phi(r) = sum M_lam^mu S_lam^{-mu}(r - r_M). Returns the real part. */
double orc_m2p(int p, const double *Min, const double *r)
{
    const cplx *M = (const cplx *)Min;
    int np = (p + 1) * (p + 1);
    cplx *S = (cplx *)malloc(sizeof(cplx) * np);
    solid_S(p, r, S);
    cplx acc = 0;
    for (int lam = 0; lam <= p; ++lam)
        for (int mu = -lam; mu <= lam; ++mu) acc += M[hidx(lam, mu)] * S[hidx(lam, -mu)];
    free(S);
    return creal(acc);
}

/* M2L with a given kernel G_j^k (j <= 2p, full index):
 *   L_l^m += sum_{lam, mu} M_lam^mu G_{l+lam}^{-(m+mu)}   (Eq. M2L / Eq. pmmm). */
static void m2l_green(int p, const cplx *M, const cplx *G, cplx *L)
{
    for (int l = 0; l <= p; ++l)
        for (int m = -l; m <= l; ++m) {
            cplx acc = 0;
            for (int lam = 0; lam <= p; ++lam)
                for (int mu = -lam; mu <= lam; ++mu) acc += M[hidx(lam, mu)] * G[hidx(l + lam, -(m + mu))];
            L[hidx(l, m)] += acc;
        }
}

void orc_m2l_green(int p, const double *M, const double *G, double *L)
{
    m2l_green(p, (const cplx *)M, (const cplx *)G, (cplx *)L);
}

/* M2L: L_l^m += sum M_lam^mu S_{l+lam}^{-(m+mu)}(r_L - r_M). */
void orc_m2l(int p, const double *M, const double *d, double *L)
{
    int ng = (2 * p + 1) * (2 * p + 1);
    cplx *G = (cplx *)malloc(sizeof(cplx) * ng);
    solid_S(2 * p, d, G);
    m2l_green(p, (const cplx *)M, G, (cplx *)L);
    free(G);
}

/* L2L: L'_l^m = sum_{lam=l..p} sum_mu L_lam^mu R_{lam-l}^{mu-m}(r_L' - r_L), for l <= pout. */
static void l2l(int p, int pout, const cplx *L, const double shift[3], cplx *Lo)
{
    int np = (p + 1) * (p + 1);
    cplx *R = (cplx *)malloc(sizeof(cplx) * np);
    solid_R(p, shift, R);
    for (int l = 0; l <= pout; ++l)
        for (int m = -l; m <= l; ++m) {
            cplx acc = 0;
            for (int lam = l; lam <= p; ++lam)
                for (int mu = -lam; mu <= lam; ++mu) {
                    int lr = lam - l, mr = mu - m;
                    if (mr < -lr || mr > lr) continue;
                    acc += L[hidx(lam, mu)] * R[hidx(lr, mr)];
                }
            Lo[hidx(l, m)] = acc;
        }
    free(R);
}

void orc_l2l(int p, int pout, const double *L, const double *shift, double *Lout)
{
    l2l(p, pout, (const cplx *)L, shift, (cplx *)Lout);
}

/* L2P: Phi(r) = sum L_lam^mu R_lam^mu(r - r_L)   (Eq. L2P), and the gradient
 * from the order-one L2L to the particle (Eq. phigrad):
 *   dPhi/dx = -Re L'_1^1,  dPhi/dy = Im L'_1^1,  dPhi/dz = L'_1^0. */
static void l2p(int p, const cplx *L, const double r[3], double *phi, double grad[3])
{
    cplx Lp[4];
    if (p >= 1) {
        l2l(p, 1, L, r, Lp);
        *phi = creal(Lp[0]);
        grad[0] = -creal(Lp[hidx(1, 1)]);
        grad[1] = cimag(Lp[hidx(1, 1)]);
        grad[2] = creal(Lp[hidx(1, 0)]);
    } else {
        *phi = creal(L[0]);
        grad[0] = grad[1] = grad[2] = 0.0;
    }
}

void orc_l2p(int p, const double *L, const double *r, double *phi, double *grad)
{
    l2p(p, (const cplx *)L, r, phi, grad);
}

/* L2P potential only, straight from Eq. L2P (used to pin the L2L route). */
double orc_l2p_phi(int p, const double *Lin, const double *r)
{
    const cplx *L = (const cplx *)Lin;
    int np = (p + 1) * (p + 1);
    cplx *R = (cplx *)malloc(sizeof(cplx) * np);
    solid_R(p, r, R);
    cplx acc = 0;
    for (int k = 0; k < np; ++k) acc += L[k] * R[k];
    free(R);
    return creal(acc);
}

/* ------------------------------------------------------------------------ */
/* Direct O(N^2) sum, open boundary: Phi_i = sum_{j != i} q_j / r_ij.        */
/* grad is the gradient of Phi at r_i.  targets: indices (or NULL = all).    */
/* ------------------------------------------------------------------------ */
void orc_direct(int64_t n, const double *pos, const double *q, int64_t nt, const int64_t *targets,
                double *phi, double *grad)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double f = 0, gx = 0, gy = 0, gz = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double ri = 1.0 / sqrt(r2);
            double qr = q[j] * ri;
            f += qr;
            double qr3 = qr * ri * ri;
            gx -= qr3 * dx;
            gy -= qr3 * dy;
            gz -= qr3 * dz;
        }
        phi[t] = f;
        grad[3 * t] = gx;
        grad[3 * t + 1] = gy;
        grad[3 * t + 2] = gz;
    }
}

/* ------------------------------------------------------------------------ */
/* Ewald sum, Eq. refewald (with q_j in the real-space line and the self term */
/* -2 alpha/sqrt(pi) q_i), rectangular box of sides box[3]:                  */
/*   real space: images with |r_ij + r_n| < rcut (j = i skipped at n = 0);    */
/*   reciprocal: k_n = (n_x/b_x, n_y/b_y, n_z/b_z), 0 < |n|_2 <= kmax.       */
/* ------------------------------------------------------------------------ */
void orc_ewald(int64_t n, const double *pos, const double *q, const double *box, double alpha, double rcut,
               double kmax, int64_t nt, const int64_t *targets, double *phi, double *grad)
{
    const double V = box[0] * box[1] * box[2];
    const double sqpi = sqrt(M_PI);
    double Q = 0;
    for (int64_t j = 0; j < n; ++j) Q += q[j];
    int nr[3];
    for (int a = 0; a < 3; ++a) nr[a] = (int)ceil(rcut / box[a]) + 1;
    int km = (int)floor(kmax);

    /* Reciprocal vectors in the half space (n_x > 0, or n_x = 0 and n_y > 0, or
     * n_x = n_y = 0 and n_z > 0); the other half is the complex conjugate. */
    int64_t nk = 0;
    for (int a = -km; a <= km; ++a)
        for (int b = -km; b <= km; ++b)
            for (int c = -km; c <= km; ++c) {
                if (a * a + b * b + c * c == 0 || a * a + b * b + c * c > kmax * kmax) continue;
                if (a > 0 || (a == 0 && (b > 0 || (b == 0 && c > 0)))) nk++;
            }
    int *kv = (int *)malloc(sizeof(int) * 3 * (nk > 0 ? nk : 1));
    cplx *Sk = (cplx *)calloc(nk > 0 ? nk : 1, sizeof(cplx));
    nk = 0;
    for (int a = -km; a <= km; ++a)
        for (int b = -km; b <= km; ++b)
            for (int c = -km; c <= km; ++c) {
                if (a * a + b * b + c * c == 0 || a * a + b * b + c * c > kmax * kmax) continue;
                if (a > 0 || (a == 0 && (b > 0 || (b == 0 && c > 0)))) {
                    kv[3 * nk] = a;
                    kv[3 * nk + 1] = b;
                    kv[3 * nk + 2] = c;
                    nk++;
                }
            }
    /* structure factors S(k) = sum_j q_j exp(2 pi i k . r_j) */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nk; ++t) {
        double k[3] = {kv[3 * t] / box[0], kv[3 * t + 1] / box[1], kv[3 * t + 2] / box[2]};
        cplx s = 0;
        for (int64_t j = 0; j < n; ++j) {
            double ph = 2.0 * M_PI * (k[0] * pos[3 * j] + k[1] * pos[3 * j + 1] + k[2] * pos[3 * j + 2]);
            s += q[j] * (cos(ph) + I * sin(ph));
        }
        Sk[t] = s;
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        const double *ri = pos + 3 * i;
        double f = 0, g[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double d0[3] = {ri[0] - pos[3 * j], ri[1] - pos[3 * j + 1], ri[2] - pos[3 * j + 2]};
            /* start from the minimum image, then scan the neighbouring images */
            for (int a = 0; a < 3; ++a) d0[a] -= box[a] * floor(d0[a] / box[a] + 0.5);
            for (int a = -nr[0]; a <= nr[0]; ++a)
                for (int b = -nr[1]; b <= nr[1]; ++b)
                    for (int c = -nr[2]; c <= nr[2]; ++c) {
                        double d[3] = {d0[0] + a * box[0], d0[1] + b * box[1], d0[2] + c * box[2]};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 >= rcut * rcut) continue;
                        if (r2 == 0.0) continue; /* j == i at n = 0 */
                        double r = sqrt(r2);
                        double e = erfc(alpha * r);
                        f += q[j] * e / r;
                        double dr = -(e / r2 + 2.0 * alpha / sqpi * exp(-alpha * alpha * r2) / r) / r;
                        for (int u = 0; u < 3; ++u) g[u] += q[j] * dr * d[u];
                    }
        }
        for (int64_t s = 0; s < nk; ++s) {
            double k[3] = {kv[3 * s] / box[0], kv[3 * s + 1] / box[1], kv[3 * s + 2] / box[2]};
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double coef = exp(-M_PI * M_PI * k2 / (alpha * alpha)) / (M_PI * V * k2);
            double ph = 2.0 * M_PI * (k[0] * ri[0] + k[1] * ri[1] + k[2] * ri[2]);
            cplx z = (cos(ph) + I * sin(ph)) * conj(Sk[s]); /* sum_j q_j exp(2 pi i k.(r_i - r_j)) */
            /* the half space carries twice the real part */
            f += 2.0 * coef * creal(z);
            for (int u = 0; u < 3; ++u) g[u] += 2.0 * coef * (-2.0 * M_PI * k[u]) * cimag(z);
        }
        f += -2.0 * alpha / sqpi * q[i] - M_PI / (V * alpha * alpha) * Q;
        phi[t] = f;
        for (int u = 0; u < 3; ++u) grad[3 * t + u] = g[u];
    }
    free(kv);
    free(Sk);
}

/* ------------------------------------------------------------------------ */
/* The same Ewald sum (Eq. refewald, same readings and truncations as        */
/* orc_ewald) for a few targets among many sources, organised so that      */
/* N = 2^20 sources stay affordable:                                        */
/*   real space: the sources are listed by cells of side >= rcut/3 (at     */
/*     least seven per axis, rcut <= 3b/7 on every axis), so a target visits */
/*     the 7^3 cells around its own; rcut < b/2 makes the minimum image the */
/*     only image within rcut;                                              */
/*   reciprocal: exp(2 pi i k.r_j) = ex^kx ey^ky ez^kz with ex = exp(2 pi i */
/*     x_j/b_x) etc., the powers taken by repeated multiplication per source */
/*     (exponential of a sum = product of exponentials); structure factors  */
/*     accumulated per thread, then summed.                                 */
/* Returns 0, or -1 when rcut > 3b/7 on some axis.                          */
/* ------------------------------------------------------------------------ */
int orc_ewald_targets(int64_t n, const double *pos, const double *q, const double *box, double alpha, double rcut,
                      double kmax, int64_t nt, const int64_t *targets, double *phi, double *grad)
{
    const double V = box[0] * box[1] * box[2];
    const double sqpi = sqrt(M_PI);
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(3.0 * box[a] / rcut);
        if (nc[a] < 7) return -1;
    }
    double Q = 0;
    for (int64_t j = 0; j < n; ++j) Q += q[j];

    /* cell list: counting sort of the sources by cell (positions wrapped into the box) */
    const int64_t NC = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *cstart = (int64_t *)calloc(NC + 1, sizeof(int64_t));
    int64_t *cidx = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *fill = (int64_t *)calloc(NC, sizeof(int64_t));
    int64_t *cellof = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) {
        int c3[3];
        for (int a = 0; a < 3; ++a) {
            double x = pos[3 * j + a] - box[a] * floor(pos[3 * j + a] / box[a]);
            int ia = (int)floor(x / box[a] * nc[a]);
            if (ia < 0) ia = 0;
            if (ia >= nc[a]) ia = nc[a] - 1;
            c3[a] = ia;
        }
        cellof[j] = c3[0] + (int64_t)nc[0] * (c3[1] + (int64_t)nc[1] * c3[2]);
        cstart[cellof[j] + 1]++;
    }
    for (int64_t c = 0; c < NC; ++c) cstart[c + 1] += cstart[c];
    for (int64_t j = 0; j < n; ++j) cidx[cstart[cellof[j]] + fill[cellof[j]]++] = j;
    /* sources copied in cell order, so that a cell's sources are read contiguously */
    double *spos = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *sq = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t u = 0; u < n; ++u) {
        for (int a = 0; a < 3; ++a) spos[3 * u + a] = pos[3 * cidx[u] + a];
        sq[u] = q[cidx[u]];
    }

    /* reciprocal vectors in the half space, as in orc_ewald */
    int km = (int)floor(kmax);
    int64_t nk = 0;
    for (int a = -km; a <= km; ++a)
        for (int b = -km; b <= km; ++b)
            for (int c = -km; c <= km; ++c) {
                if (a * a + b * b + c * c == 0 || a * a + b * b + c * c > kmax * kmax) continue;
                if (a > 0 || (a == 0 && (b > 0 || (b == 0 && c > 0)))) nk++;
            }
    int *kv = (int *)malloc(sizeof(int) * 3 * (nk > 0 ? nk : 1));
    cplx *Sk = (cplx *)calloc(nk > 0 ? nk : 1, sizeof(cplx));
    nk = 0;
    for (int a = -km; a <= km; ++a)
        for (int b = -km; b <= km; ++b)
            for (int c = -km; c <= km; ++c) {
                if (a * a + b * b + c * c == 0 || a * a + b * b + c * c > kmax * kmax) continue;
                if (a > 0 || (a == 0 && (b > 0 || (b == 0 && c > 0)))) {
                    kv[3 * nk] = a;
                    kv[3 * nk + 1] = b;
                    kv[3 * nk + 2] = c;
                    nk++;
                }
            }
    /* structure factors S(k) = sum_j q_j exp(2 pi i k . r_j), sources taken in
     * blocks of SB (their phase factors ep[j][axis][m] = exp(2 pi i m x/b), m in
     * [-km, km]); kv lists the vectors with kx, then ky, then kz increasing, so
     * q_j ex^kx ey^ky is formed once per (kx, ky) run */
    enum { SB = 256 };
    const int W = 2 * km + 1;
#pragma omp parallel
    {
        cplx *Sl = (cplx *)calloc(nk > 0 ? nk : 1, sizeof(cplx));
        cplx *ep = (cplx *)malloc(sizeof(cplx) * SB * 3 * W);
#pragma omp for schedule(static)
        for (int64_t j0 = 0; j0 < n; j0 += SB) {
            const int nb = (int)(n - j0 < SB ? n - j0 : SB);
            for (int jj = 0; jj < nb; ++jj)
                for (int a = 0; a < 3; ++a) {
                    cplx *e = ep + ((int64_t)jj * 3 + a) * W;
                    double ph = 2.0 * M_PI * pos[3 * (j0 + jj) + a] / box[a];
                    cplx w = cos(ph) + I * sin(ph);
                    e[km] = 1.0;
                    for (int m = 1; m <= km; ++m) {
                        e[km + m] = e[km + m - 1] * w;
                        e[km - m] = conj(e[km + m]);
                    }
                }
            int64_t t = 0;
            while (t < nk) {
                const int a = kv[3 * t], b = kv[3 * t + 1];
                int64_t t1 = t;
                while (t1 < nk && kv[3 * t1] == a && kv[3 * t1 + 1] == b) ++t1;
                for (int jj = 0; jj < nb; ++jj) {
                    const cplx *e = ep + (int64_t)jj * 3 * W;
                    const cplx qxy = q[j0 + jj] * (e[km + a] * e[W + km + b]);
                    for (int64_t u = t; u < t1; ++u) Sl[u] += qxy * e[2 * W + km + kv[3 * u + 2]];
                }
                t = t1;
            }
        }
#pragma omp critical
        for (int64_t t = 0; t < nk; ++t) Sk[t] += Sl[t];
        free(ep);
        free(Sl);
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        const double *ri = pos + 3 * i;
        double f = 0, g[3] = {0, 0, 0};
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            double x = ri[a] - box[a] * floor(ri[a] / box[a]);
            ci[a] = (int)floor(x / box[a] * nc[a]);
            if (ci[a] < 0) ci[a] = 0;
            if (ci[a] >= nc[a]) ci[a] = nc[a] - 1;
        }
        for (int dz = -3; dz <= 3; ++dz)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx) {
                    int cx = (ci[0] + dx + nc[0]) % nc[0], cy = (ci[1] + dy + nc[1]) % nc[1],
                        cz = (ci[2] + dz + nc[2]) % nc[2];
                    int64_t c = cx + (int64_t)nc[0] * (cy + (int64_t)nc[1] * cz);
                    for (int64_t u = cstart[c]; u < cstart[c + 1]; ++u) {
                        const double *rj = spos + 3 * u;
                        double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
                        for (int a = 0; a < 3; ++a) d[a] -= box[a] * floor(d[a] / box[a] + 0.5);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 >= rcut * rcut) continue;
                        if (r2 == 0.0) continue; /* j == i */
                        double r = sqrt(r2);
                        double ec = erfc(alpha * r);
                        f += sq[u] * ec / r;
                        double dr = -(ec / r2 + 2.0 * alpha / sqpi * exp(-alpha * alpha * r2) / r) / r;
                        for (int a = 0; a < 3; ++a) g[a] += sq[u] * dr * d[a];
                    }
                }
        for (int64_t s = 0; s < nk; ++s) {
            double k[3] = {kv[3 * s] / box[0], kv[3 * s + 1] / box[1], kv[3 * s + 2] / box[2]};
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double coef = exp(-M_PI * M_PI * k2 / (alpha * alpha)) / (M_PI * V * k2);
            double ph = 2.0 * M_PI * (k[0] * ri[0] + k[1] * ri[1] + k[2] * ri[2]);
            cplx z = (cos(ph) + I * sin(ph)) * conj(Sk[s]);
            f += 2.0 * coef * creal(z);
            for (int a = 0; a < 3; ++a) g[a] += 2.0 * coef * (-2.0 * M_PI * k[a]) * cimag(z);
        }
        f += -2.0 * alpha / sqpi * q[i] - M_PI / (V * alpha * alpha) * Q;
        phi[t] = f;
        for (int a = 0; a < 3; ++a) grad[3 * t + a] = g[a];
    }
    free(kv);
    free(Sk);
    free(cstart);
    free(cidx);
    free(fill);
    free(cellof);
    free(spos);
    free(sq);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Binning (Sec. 2.1: particles assigned to K uniform cells in O(N)).        */
/* The FP64 formula, in this order, each operation rounded:                  */
/*   t = x - lo;  if t is outside [0, len):                                  */
/*     periodic: t = t - len * floor(t / len), if t >= len: t -= len         */
/*     open: error                                                           */
/*   i = floor(t * inv) with inv = n / len, clamped to [0, n-1]              */
/* Cell id = ix + nx * (iy + ny * iz).  Stable counting sort by cell id:     */
/* perm lists original indices in (cell, original index) order.              */
/* Returns 0, or -3 for a particle outside the open box / -4 non-finite.     */
/* wrapped (optional, n*3): the coordinate lo + t actually binned.           */
/* ------------------------------------------------------------------------ */
int orc_bin(int64_t n, const double *pos, const double *lo, const double *len, const int *mesh, int periodic,
            int32_t *cell, int64_t *perm, int64_t *cell_start, double *wrapped)
{
    int status = 0;
    int64_t K = (int64_t)mesh[0] * mesh[1] * mesh[2];
    double inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = (double)mesh[a] / len[a];
    for (int64_t i = 0; i < n; ++i) {
        int ix[3];
        for (int a = 0; a < 3; ++a) {
            double x = pos[3 * i + a];
            if (!isfinite(x)) {
                if (status == 0) status = -4;
                ix[a] = 0;
                if (wrapped) wrapped[3 * i + a] = lo[a];
                continue;
            }
            volatile double t = x - lo[a];
            if (!(t >= 0.0 && t < len[a])) {
                if (periodic) {
                    volatile double qd = t / len[a];
                    volatile double fl = floor(qd);
                    volatile double w = len[a] * fl;
                    t = t - w;
                    if (t >= len[a]) t = t - len[a];
                } else if (status == 0) {
                    status = -3;
                }
            }
            volatile double s = t * inv[a];
            double f = floor(s);
            int k;
            if (f < 0.0) k = 0;
            else if (f > (double)(mesh[a] - 1)) k = mesh[a] - 1;
            else k = (int)f;
            ix[a] = k;
            if (wrapped) wrapped[3 * i + a] = lo[a] + t;
        }
        cell[i] = (int32_t)(ix[0] + (int64_t)mesh[0] * (ix[1] + (int64_t)mesh[1] * ix[2]));
    }
    /* stable counting sort */
    for (int64_t c = 0; c <= K; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) cell_start[cell[i] + 1]++;
    for (int64_t c = 0; c < K; ++c) cell_start[c + 1] += cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (K > 0 ? K : 1));
    for (int64_t c = 0; c < K; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[cell[i]]++] = i;
    free(fill);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Green functions.  G holds (2p+1)^2 complex values G_j^k, j <= 2p, full    */
/* index, so that the M2L of cell j to cell i is                              */
/*   L_l^m += sum M_lam^mu G_{l+lam}^{-(m+mu)}(i - j).                        */
/* ------------------------------------------------------------------------ */

/* Open boundary (Sec. 2.1 mask, App. C): S_j^k(d h) for |d|_inf > c, else 0.
 * d is the cell displacement i - j (no wrap), h the cell size per axis. */
void orc_green_open(int p, int c, const double *h, const int *d, double *Gout)
{
    cplx *G = (cplx *)Gout;
    int ng = (2 * p + 1) * (2 * p + 1);
    int dm = abs(d[0]);
    if (abs(d[1]) > dm) dm = abs(d[1]);
    if (abs(d[2]) > dm) dm = abs(d[2]);
    if (dm <= c) {
        for (int k = 0; k < ng; ++k) G[k] = 0;
        return;
    }
    double r[3] = {d[0] * h[0], d[1] * h[1], d[2] * h[2]};
    solid_S(2 * p, r, G);
}

/* Periodic boundary (App. B): the lattice sum of S over all images, by the
 * Ewald split of Eq. greenPBC with splitting parameter alpha, both sums over
 * |n|_2 <= nmax, minus the one image whose cell offset has |.|_inf <= c
 * (masked; handled by the near field).  The masked image enters the split as
 * -P(j+1/2, (alpha r)^2) S_j instead of Q(j+1/2, (alpha r)^2) S_j; the masked
 * image at zero offset (the self cell) is left out entirely; its l = 0 limit
 * is the -2 alpha/sqrt(pi) M_0^0 term of the correction procedure.
 * d is any cell offset; the minimum-image representative is used. */
void orc_green_periodic(int p, int c, const int *mesh, const double *box, double alpha, int nmax, const int *d,
                        double *Gout)
{
    cplx *G = (cplx *)Gout;
    int J = 2 * p;
    int ng = (J + 1) * (J + 1);
    double h[3], V = box[0] * box[1] * box[2];
    int dm[3];
    for (int a = 0; a < 3; ++a) {
        h[a] = box[a] / mesh[a];
        int v = ((d[a] % mesh[a]) + mesh[a]) % mesh[a];
        if (2 * v > mesh[a]) v -= mesh[a];
        dm[a] = v;
    }
    for (int k = 0; k < ng; ++k) G[k] = 0;
    cplx *S = (cplx *)malloc(sizeof(cplx) * ng);
    double r0[3] = {dm[0] * h[0], dm[1] * h[1], dm[2] * h[2]};

    /* real-space part */
    for (int a = -nmax; a <= nmax; ++a)
        for (int b = -nmax; b <= nmax; ++b)
            for (int e = -nmax; e <= nmax; ++e) {
                if (a * a + b * b + e * e > nmax * nmax) continue;
                int D[3] = {dm[0] + a * mesh[0], dm[1] + b * mesh[1], dm[2] + e * mesh[2]};
                int near = abs(D[0]) <= c && abs(D[1]) <= c && abs(D[2]) <= c;
                if (near && D[0] == 0 && D[1] == 0 && D[2] == 0) continue;
                double rv[3] = {r0[0] + a * box[0], r0[1] + b * box[1], r0[2] + e * box[2]};
                double r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
                double x = alpha * alpha * r2;
                solid_S(J, rv, S);
                for (int j = 0; j <= J; ++j) {
                    double w = near ? -orc_gammaP_half(j, x) : orc_gammaQ_half(j, x);
                    for (int k = -j; k <= j; ++k) G[hidx(j, k)] += w * S[hidx(j, k)];
                }
            }
    /* reciprocal part */
    for (int a = -nmax; a <= nmax; ++a)
        for (int b = -nmax; b <= nmax; ++b)
            for (int e = -nmax; e <= nmax; ++e) {
                int nn = a * a + b * b + e * e;
                if (nn == 0 || nn > nmax * nmax) continue;
                double kv[3] = {a / box[0], b / box[1], e / box[2]};
                double kk = sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
                solid_S(J, kv, S);
                double ph = 2.0 * M_PI * (kv[0] * r0[0] + kv[1] * r0[1] + kv[2] * r0[2]);
                cplx phase = cos(ph) + I * sin(ph);
                double g = exp(-(M_PI * kk / alpha) * (M_PI * kk / alpha));
                cplx mipi = 1.0; /* (-i pi)^j */
                for (int j = 0; j <= J; ++j) {
                    cplx coef = mipi / sqrt(M_PI) * g / tgamma(j + 0.5) * pow(kk, 2.0 * j - 1.0) / V;
                    for (int k = -j; k <= j; ++k) G[hidx(j, k)] += coef * S[hidx(j, k)] * phase;
                    mipi *= -I * M_PI;
                }
            }
    free(S);
}

/* ------------------------------------------------------------------------ */
/* PMMM by its definition (Sec. 2.1, Eq. pmmm): L_i = sum_j G_{i-j} M_j over  */
/* all cell pairs, then the corrections (periodic, App. B.3), L2P with the   */
/* order-one L2L gradient, and the near field over the (2c+1)^3 masked cells. */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], len[3];
    int mesh[3];
    int p, c, periodic;
    double alpha;
    int nmax;
} orc_cfg;

/* Returns 0 or a binning error.  For each target cell in tcells (all cells if
 * ntc < 0), writes phi / grad (gradient of Phi, Coulomb sign) of its
 * particles at their ORIGINAL indices; other entries are left untouched.
 * M_out (K * (p+1)^2 complex, optional): multipoles of all cells.
 * L_out (K * (p+1)^2 complex, optional): local expansions of target cells
 *   after the cell convolution, before the corrections.
 * corr_out (8 doubles, optional): Q, sum_cells M_1^0, Re/Im sum_cells M_1^1,
 *   sum q|r_rel|^2, and 3 spare. */
/* Number of distinct cell displacements of the Green-function table and its
 * dimensions: n^3 (periodic, d mod n) or (2n-1)^3 (open, d in [-(n-1), n-1]). */
int64_t orc_green_table_size(const orc_cfg *cfg)
{
    int gx = cfg->periodic ? cfg->mesh[0] : 2 * cfg->mesh[0] - 1;
    int gy = cfg->periodic ? cfg->mesh[1] : 2 * cfg->mesh[1] - 1;
    int gz = cfg->periodic ? cfg->mesh[2] : 2 * cfg->mesh[2] - 1;
    return (int64_t)gx * gy * gz;
}

/* The Green function of every distinct displacement, (2p+1)^2 complex values
 * each (Sec. 2.1: computed once at the beginning and saved). */
void orc_green_table(const orc_cfg *cfg, double *out)
{
    const int p = cfg->p, c = cfg->c;
    const int nx = cfg->mesh[0], ny = cfg->mesh[1], nz = cfg->mesh[2];
    const int ng = (2 * p + 1) * (2 * p + 1);
    double h[3];
    for (int a = 0; a < 3; ++a) h[a] = cfg->len[a] / cfg->mesh[a];
    int gx = cfg->periodic ? nx : 2 * nx - 1, gy = cfg->periodic ? ny : 2 * ny - 1;
    int64_t NG = orc_green_table_size(cfg);
    cplx *Gall = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < NG; ++t) {
        int a = (int)(t % gx), b = (int)((t / gx) % gy), e = (int)(t / ((int64_t)gx * gy));
        if (cfg->periodic) {
            int d[3] = {a, b, e};
            orc_green_periodic(p, c, cfg->mesh, cfg->len, cfg->alpha, cfg->nmax, d, (double *)(Gall + t * ng));
        } else {
            int d[3] = {a - (nx - 1), b - (ny - 1), e - (nz - 1)};
            orc_green_open(p, c, h, d, (double *)(Gall + t * ng));
        }
    }
}

/* Near field of particle i (binned position wp[3i], in cell (ix, iy, iz) of
 * cfg's mesh): pure 1/r over the particles of the (2c+1)^3 masked cells
 * (Sec. 2.1), periodic neighbours shifted by a box length; adds to *f and g
 * (gradient of Phi). */
static void near_field(const orc_cfg *cfg, const int64_t *cs, const int64_t *perm, const double *wp,
                       const double *q, int64_t i, int ix, int iy, int iz, double *f, double g[3])
{
    const int c = cfg->c, nx = cfg->mesh[0], ny = cfg->mesh[1], nz = cfg->mesh[2];
    const double *ri = wp + 3 * i;
    for (int ez = -c; ez <= c; ++ez)
        for (int ey = -c; ey <= c; ++ey)
            for (int ex = -c; ex <= c; ++ex) {
                int jx = ix + ex, jy = iy + ey, jz = iz + ez;
                double sh[3] = {0, 0, 0};
                if (cfg->periodic) {
                    int wx = ((jx % nx) + nx) % nx, wy = ((jy % ny) + ny) % ny, wz = ((jz % nz) + nz) % nz;
                    sh[0] = (double)((jx - wx) / nx) * cfg->len[0];
                    sh[1] = (double)((jy - wy) / ny) * cfg->len[1];
                    sh[2] = (double)((jz - wz) / nz) * cfg->len[2];
                    jx = wx; jy = wy; jz = wz;
                } else if (jx < 0 || jy < 0 || jz < 0 || jx >= nx || jy >= ny || jz >= nz) {
                    continue;
                }
                int64_t cj = jx + (int64_t)nx * (jy + (int64_t)ny * jz);
                for (int64_t u = cs[cj]; u < cs[cj + 1]; ++u) {
                    int64_t j = perm[u];
                    if (j == i) continue;
                    double d[3] = {ri[0] - (wp[3 * j] + sh[0]), ri[1] - (wp[3 * j + 1] + sh[1]),
                                   ri[2] - (wp[3 * j + 2] + sh[2])};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 == 0.0) continue;
                    double rinv = 1.0 / sqrt(r2);
                    *f += q[j] * rinv;
                    for (int a = 0; a < 3; ++a) g[a] -= q[j] * rinv * rinv * rinv * d[a];
                }
            }
}

/* green_table: optional table from orc_green_table for the same cfg (not owned). */
int orc_pmmm(const orc_cfg *cfg, int64_t n, const double *pos, const double *q, int64_t ntc, const int64_t *tcells,
             double *phi, double *grad, double *M_out, double *L_out, double *corr_out, const double *green_table)
{
    const int p = cfg->p, c = cfg->c, J = 2 * p;
    const int nx = cfg->mesh[0], ny = cfg->mesh[1], nz = cfg->mesh[2];
    const int64_t K = (int64_t)nx * ny * nz;
    const int np = (p + 1) * (p + 1), ng = (J + 1) * (J + 1);
    double h[3], V = cfg->len[0] * cfg->len[1] * cfg->len[2];
    for (int a = 0; a < 3; ++a) h[a] = cfg->len[a] / cfg->mesh[a];

    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *cs = (int64_t *)malloc(sizeof(int64_t) * (K + 1));
    double *wp = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    int st = orc_bin(n, pos, cfg->lo, cfg->len, cfg->mesh, cfg->periodic, cell, perm, cs, wp);
    if (st != 0) {
        free(cell); free(perm); free(cs); free(wp);
        return st;
    }

    /* cell centres and relative positions */
    cplx *M = (cplx *)calloc((size_t)K * np, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t ci = 0; ci < K; ++ci) {
        int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
        double ctr[3] = {cfg->lo[0] + (ix + 0.5) * h[0], cfg->lo[1] + (iy + 0.5) * h[1], cfg->lo[2] + (iz + 0.5) * h[2]};
        for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
            int64_t i = perm[s];
            p2m(p, 1, wp + 3 * i, q + i, ctr, M + ci * np);
        }
    }
    if (M_out) memcpy(M_out, M, sizeof(cplx) * K * np);

    /* Green function for every distinct displacement, precomputed when that
     * table fits in 1 GiB, else evaluated for each cell pair. */
    int gx = cfg->periodic ? nx : 2 * nx - 1, gy = cfg->periodic ? ny : 2 * ny - 1, gz = cfg->periodic ? nz : 2 * nz - 1;
    int64_t NG = (int64_t)gx * gy * gz;
    int owned = !green_table && (double)NG * ng * sizeof(cplx) <= (double)(1 << 30);
    int table = green_table != NULL || owned;
    cplx *Gall = NULL;
    if (green_table) {
        Gall = (cplx *)green_table;
    } else if (owned) {
        Gall = (cplx *)malloc(sizeof(cplx) * NG * ng);
        orc_green_table(cfg, (double *)Gall);
    }

    int64_t nT = ntc < 0 ? K : ntc;
    cplx *L = (cplx *)calloc((size_t)nT * np, sizeof(cplx));
#pragma omp parallel
    {
        cplx *Gp = (cplx *)malloc(sizeof(cplx) * ng);
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < nT; ++t) {
            int64_t ci = ntc < 0 ? t : tcells[t];
            int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
            for (int64_t cj = 0; cj < K; ++cj) {
                int jx = (int)(cj % nx), jy = (int)((cj / nx) % ny), jz = (int)(cj / ((int64_t)nx * ny));
                const cplx *G;
                if (cfg->periodic) {
                    int d[3] = {((ix - jx) % nx + nx) % nx, ((iy - jy) % ny + ny) % ny, ((iz - jz) % nz + nz) % nz};
                    if (table) {
                        G = Gall + (d[0] + (int64_t)gx * (d[1] + (int64_t)gy * d[2])) * ng;
                    } else {
                        orc_green_periodic(p, c, cfg->mesh, cfg->len, cfg->alpha, cfg->nmax, d, (double *)Gp);
                        G = Gp;
                    }
                } else {
                    int d[3] = {ix - jx, iy - jy, iz - jz};
                    if (table) {
                        G = Gall + ((d[0] + nx - 1) + (int64_t)gx * ((d[1] + ny - 1) + (int64_t)gy * (d[2] + nz - 1))) * ng;
                    } else {
                        orc_green_open(p, c, h, d, (double *)Gp);
                        G = Gp;
                    }
                }
                m2l_green(p, M + cj * np, G, L + t * np);
            }
        }
        free(Gp);
    }
    if (owned) free(Gall);
    if (L_out)
        for (int64_t t = 0; t < nT; ++t) {
            int64_t ci = ntc < 0 ? t : tcells[t];
            memcpy(L_out + 2 * ci * np, L + t * np, sizeof(cplx) * np);
        }

    /* periodic corrections (App. B.3) */
    double Qtot = 0, q2sum = 0;
    cplx sM10 = 0, sM11 = 0;
    for (int64_t i = 0; i < n; ++i) Qtot += q[i];
    if (cfg->periodic) {
        for (int64_t ci = 0; ci < K; ++ci) {
            if (p >= 1) {
                sM10 += M[ci * np + hidx(1, 0)];
                sM11 += M[ci * np + hidx(1, 1)];
            }
        }
        for (int64_t ci = 0; ci < K; ++ci) {
            int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
            double ctr[3] = {cfg->lo[0] + (ix + 0.5) * h[0], cfg->lo[1] + (iy + 0.5) * h[1], cfg->lo[2] + (iz + 0.5) * h[2]};
            for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
                int64_t i = perm[s];
                double rr = 0;
                for (int a = 0; a < 3; ++a) rr += (wp[3 * i + a] - ctr[a]) * (wp[3 * i + a] - ctr[a]);
                q2sum += q[i] * rr;
            }
        }
        for (int64_t t = 0; t < nT; ++t) {
            int64_t ci = ntc < 0 ? t : tcells[t];
            cplx *Lc = L + t * np;
            if (p >= 1) {
                Lc[hidx(1, 0)] += 4.0 * M_PI / (3.0 * V) * sM10;
                cplx d11 = 8.0 * M_PI / (3.0 * V) * conj(sM11);
                Lc[hidx(1, 1)] += d11;
                Lc[hidx(1, -1)] += -conj(d11); /* keeps L_1^{-1} = -conj(L_1^1) */
            }
            Lc[0] += -2.0 * cfg->alpha / sqrt(M_PI) * M[ci * np] + 2.0 * M_PI / (3.0 * V) * q2sum;
        }
    }
    if (corr_out) {
        corr_out[0] = Qtot;
        corr_out[1] = creal(sM10);
        corr_out[2] = creal(sM11);
        corr_out[3] = cimag(sM11);
        corr_out[4] = q2sum;
        corr_out[5] = corr_out[6] = corr_out[7] = 0;
    }

    /* L2P + near field for the particles of the target cells */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nT; ++t) {
        int64_t ci = ntc < 0 ? t : tcells[t];
        int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
        double ctr[3] = {cfg->lo[0] + (ix + 0.5) * h[0], cfg->lo[1] + (iy + 0.5) * h[1], cfg->lo[2] + (iz + 0.5) * h[2]};
        for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
            int64_t i = perm[s];
            const double *ri = wp + 3 * i;
            double rel[3] = {ri[0] - ctr[0], ri[1] - ctr[1], ri[2] - ctr[2]};
            double f, g[3];
            l2p(p, L + t * np, rel, &f, g);
            if (cfg->periodic && Qtot != 0.0) {
                double rr = rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2];
                f += 2.0 * M_PI / (3.0 * V) * Qtot * (rr - 3.0 / (2.0 * cfg->alpha * cfg->alpha));
                for (int a = 0; a < 3; ++a) g[a] += 4.0 * M_PI / (3.0 * V) * Qtot * rel[a];
            }
            near_field(cfg, cs, perm, wp, q, i, ix, iy, iz, &f, g);
            phi[i] = f;
            for (int a = 0; a < 3; ++a) grad[3 * i + a] = g[a];
        }
    }

    free(L);
    free(M);
    free(cell);
    free(perm);
    free(cs);
    free(wp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-level PMMM (Sec. 5, hierarchical treatment; Fig. refine).             */
/*                                                                          */
/* The mesh of cfg is the fine mesh; every `refine`^3 block of fine cells is */
/* one coarse cell.  By the definition of the method:                       */
/*  1. coarse level: PMMM on the coarse mesh (coarse multipoles by Eq. P2M  */
/*     at the coarse centres, L_T = sum_S G(T - S) M_S over all coarse     */
/*     pairs with the coarse Green function, whose nearest (2c+1)^3 coarse */
/*     cells are masked), with the periodic corrections of App. B.3 taken  */
/*     at the coarse level (coarse-cell-relative positions, coarse M_0^0);  */
/*  2. fine level: every fine source cell s whose coarse cell S lies in the */
/*     masked (2c+1)^3 block of the target's coarse cell T contributes      */
/*     M2L(M_s, r_t - r_s) with the free-space kernel, unless the fine      */
/*     cells are themselves nearest neighbours (|t - s|_inf <= c);          */
/*  3. the rest, the fine (2c+1)^3 near cells, by the direct 1/r sum.      */
/* The potential of a particle is the coarse local expansion evaluated at   */
/* its offset from the coarse centre (Eq. L2P, with the order-one L2L       */
/* gradient) plus the fine local expansion at its offset from the fine      */
/* centre plus its near field.                                              */
/*                                                                          */
/* M_out (K_fine * (p+1)^2 complex, optional): fine multipoles.             */
/* L_out (optional): for each target fine cell t, the total local expansion */
/* before the periodic corrections, as one fine-centred expansion:          */
/* L2L(L_T, r_t - r_T) + the fine-level sum.                                */
/* green_coarse (optional): orc_green_table of the coarse geometry.         */
/* ------------------------------------------------------------------------ */
int orc_pmmm_hier(const orc_cfg *cfg, int refine, int64_t n, const double *pos, const double *q, int64_t ntc,
                  const int64_t *tcells, double *phi, double *grad, double *M_out, double *L_out,
                  const double *green_coarse)
{
    const int p = cfg->p, c = cfg->c, r = refine, J = 2 * p;
    const int np = (p + 1) * (p + 1), ng = (J + 1) * (J + 1);
    if (r < 1) return -1;
    for (int a = 0; a < 3; ++a)
        if (cfg->mesh[a] % r != 0) return -1;
    const int nx = cfg->mesh[0], ny = cfg->mesh[1], nz = cfg->mesh[2];
    const int64_t K = (int64_t)nx * ny * nz;
    orc_cfg cc = *cfg;
    for (int a = 0; a < 3; ++a) cc.mesh[a] = cfg->mesh[a] / r;
    const int mx = cc.mesh[0], my = cc.mesh[1], mz = cc.mesh[2];
    const int64_t Kc = (int64_t)mx * my * mz;
    double hf[3], hc[3], V = cfg->len[0] * cfg->len[1] * cfg->len[2];
    for (int a = 0; a < 3; ++a) {
        hf[a] = cfg->len[a] / cfg->mesh[a];
        hc[a] = hf[a] * r;
    }

    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *cs = (int64_t *)malloc(sizeof(int64_t) * (K + 1));
    double *wp = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    int st = orc_bin(n, pos, cfg->lo, cfg->len, cfg->mesh, cfg->periodic, cell, perm, cs, wp);
    if (st != 0) {
        free(cell); free(perm); free(cs); free(wp);
        return st;
    }

    /* fine and coarse multipoles (Eq. P2M at the fine and at the coarse centres) */
    cplx *Mf = (cplx *)calloc((size_t)K * np, sizeof(cplx));
    cplx *Mc = (cplx *)calloc((size_t)Kc * np, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t ci = 0; ci < K; ++ci) {
        int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
        double ctr[3] = {cfg->lo[0] + (ix + 0.5) * hf[0], cfg->lo[1] + (iy + 0.5) * hf[1],
                         cfg->lo[2] + (iz + 0.5) * hf[2]};
        for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
            int64_t i = perm[s];
            p2m(p, 1, wp + 3 * i, q + i, ctr, Mf + ci * np);
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t T = 0; T < Kc; ++T) {
        int Tx = (int)(T % mx), Ty = (int)((T / mx) % my), Tz = (int)(T / ((int64_t)mx * my));
        double ctr[3] = {cfg->lo[0] + (Tx + 0.5) * hc[0], cfg->lo[1] + (Ty + 0.5) * hc[1],
                         cfg->lo[2] + (Tz + 0.5) * hc[2]};
        for (int bz = 0; bz < r; ++bz)
            for (int by = 0; by < r; ++by)
                for (int bx = 0; bx < r; ++bx) {
                    int64_t ci = (Tx * r + bx) + (int64_t)nx * ((Ty * r + by) + (int64_t)ny * (Tz * r + bz));
                    for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
                        int64_t i = perm[s];
                        p2m(p, 1, wp + 3 * i, q + i, ctr, Mc + T * np);
                    }
                }
    }
    if (M_out) memcpy(M_out, Mf, sizeof(cplx) * K * np);

    /* target fine cells and the coarse cells they lie in */
    int64_t nT = ntc < 0 ? K : ntc;
    char *need = (char *)calloc((size_t)Kc, 1);
    for (int64_t t = 0; t < nT; ++t) {
        int64_t ci = ntc < 0 ? t : tcells[t];
        int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
        need[(ix / r) + (int64_t)mx * ((iy / r) + (int64_t)my * (iz / r))] = 1;
    }

    /* coarse level: cell-pair convolution with the coarse Green function */
    int gx = cc.periodic ? mx : 2 * mx - 1, gy = cc.periodic ? my : 2 * my - 1, gz = cc.periodic ? mz : 2 * mz - 1;
    int64_t NG = (int64_t)gx * gy * gz;
    cplx *Gc = (cplx *)green_coarse;
    int owned = 0;
    if (!Gc) {
        Gc = (cplx *)malloc(sizeof(cplx) * NG * ng);
        orc_green_table(&cc, (double *)Gc);
        owned = 1;
    }
    cplx *Lc = (cplx *)calloc((size_t)Kc * np, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t T = 0; T < Kc; ++T) {
        if (!need[T]) continue;
        int Tx = (int)(T % mx), Ty = (int)((T / mx) % my), Tz = (int)(T / ((int64_t)mx * my));
        for (int64_t S = 0; S < Kc; ++S) {
            int Sx = (int)(S % mx), Sy = (int)((S / mx) % my), Sz = (int)(S / ((int64_t)mx * my));
            int64_t gi;
            if (cc.periodic) {
                int d[3] = {((Tx - Sx) % mx + mx) % mx, ((Ty - Sy) % my + my) % my, ((Tz - Sz) % mz + mz) % mz};
                gi = d[0] + (int64_t)gx * (d[1] + (int64_t)gy * d[2]);
            } else {
                gi = (Tx - Sx + mx - 1) + (int64_t)gx * ((Ty - Sy + my - 1) + (int64_t)gy * (Tz - Sz + mz - 1));
            }
            m2l_green(p, Mc + S * np, Gc + gi * ng, Lc + T * np);
        }
    }
    if (owned) free(Gc);
    cplx *Lc0 = (cplx *)malloc(sizeof(cplx) * (size_t)Kc * np);
    memcpy(Lc0, Lc, sizeof(cplx) * (size_t)Kc * np);

    /* periodic corrections (App. B.3) at the coarse level */
    double Qtot = 0, q2sum = 0;
    for (int64_t i = 0; i < n; ++i) Qtot += q[i];
    if (cfg->periodic) {
        cplx sM10 = 0, sM11 = 0;
        for (int64_t T = 0; T < Kc; ++T) {
            if (p >= 1) {
                sM10 += Mc[T * np + hidx(1, 0)];
                sM11 += Mc[T * np + hidx(1, 1)];
            }
        }
        for (int64_t ci = 0; ci < K; ++ci) {
            int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
            double ctr[3] = {cfg->lo[0] + (ix / r + 0.5) * hc[0], cfg->lo[1] + (iy / r + 0.5) * hc[1],
                             cfg->lo[2] + (iz / r + 0.5) * hc[2]};
            for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
                int64_t i = perm[s];
                double rr = 0;
                for (int a = 0; a < 3; ++a) rr += (wp[3 * i + a] - ctr[a]) * (wp[3 * i + a] - ctr[a]);
                q2sum += q[i] * rr;
            }
        }
        for (int64_t T = 0; T < Kc; ++T) {
            if (!need[T]) continue;
            cplx *L = Lc + T * np;
            if (p >= 1) {
                L[hidx(1, 0)] += 4.0 * M_PI / (3.0 * V) * sM10;
                cplx d11 = 8.0 * M_PI / (3.0 * V) * conj(sM11);
                L[hidx(1, 1)] += d11;
                L[hidx(1, -1)] += -conj(d11);
            }
            L[0] += -2.0 * cfg->alpha / sqrt(M_PI) * Mc[T * np] + 2.0 * M_PI / (3.0 * V) * q2sum;
        }
    }

    /* fine level: free-space kernel of every fine offset the masked coarse block can hold */
    const int D = (c + 1) * r - 1, W = 2 * D + 1;
    cplx *Gf = (cplx *)malloc(sizeof(cplx) * (size_t)W * W * W * ng);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t u = 0; u < (int64_t)W * W * W; ++u) {
        int d[3] = {(int)(u % W) - D, (int)((u / W) % W) - D, (int)(u / ((int64_t)W * W)) - D};
        orc_green_open(p, c, hf, d, (double *)(Gf + u * ng));
    }
    cplx *Lf = (cplx *)calloc((size_t)nT * np, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nT; ++t) {
        int64_t ci = ntc < 0 ? t : tcells[t];
        int tx = (int)(ci % nx), ty = (int)((ci / nx) % ny), tz = (int)(ci / ((int64_t)nx * ny));
        int T3[3] = {tx / r, ty / r, tz / r}, A3[3] = {tx % r, ty % r, tz % r};
        for (int ez = -c; ez <= c; ++ez)
            for (int ey = -c; ey <= c; ++ey)
                for (int ex = -c; ex <= c; ++ex) {
                    int E3[3] = {ex, ey, ez}, S3[3];
                    int skip = 0;
                    for (int a = 0; a < 3; ++a) {
                        S3[a] = T3[a] + E3[a];
                        if (S3[a] < 0 || S3[a] >= cc.mesh[a]) {
                            if (!cfg->periodic) skip = 1;
                            S3[a] = ((S3[a] % cc.mesh[a]) + cc.mesh[a]) % cc.mesh[a];
                        }
                    }
                    if (skip) continue;
                    for (int bz = 0; bz < r; ++bz)
                        for (int by = 0; by < r; ++by)
                            for (int bx = 0; bx < r; ++bx) {
                                int B3[3] = {bx, by, bz}, d[3];
                                for (int a = 0; a < 3; ++a) d[a] = A3[a] - B3[a] - E3[a] * r;
                                int64_t sc = (S3[0] * r + bx) + (int64_t)nx * ((S3[1] * r + by) +
                                                                                (int64_t)ny * (S3[2] * r + bz));
                                int64_t u = (d[0] + D) + (int64_t)W * ((d[1] + D) + (int64_t)W * (d[2] + D));
                                m2l_green(p, Mf + sc * np, Gf + u * ng, Lf + t * np);
                            }
                }
    }
    free(Gf);

    if (L_out)
        for (int64_t t = 0; t < nT; ++t) {
            int64_t ci = ntc < 0 ? t : tcells[t];
            int tx = (int)(ci % nx), ty = (int)((ci / nx) % ny), tz = (int)(ci / ((int64_t)nx * ny));
            int64_t T = (tx / r) + (int64_t)mx * ((ty / r) + (int64_t)my * (tz / r));
            double sh[3] = {((tx % r) + 0.5) * hf[0] - 0.5 * hc[0], ((ty % r) + 0.5) * hf[1] - 0.5 * hc[1],
                            ((tz % r) + 0.5) * hf[2] - 0.5 * hc[2]};
            cplx *Lo = (cplx *)L_out + ci * np;
            l2l(p, p, Lc0 + T * np, sh, Lo);
            for (int k = 0; k < np; ++k) Lo[k] += Lf[t * np + k];
        }

    /* potential and gradient of the particles of the target cells */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nT; ++t) {
        int64_t ci = ntc < 0 ? t : tcells[t];
        int ix = (int)(ci % nx), iy = (int)((ci / nx) % ny), iz = (int)(ci / ((int64_t)nx * ny));
        int64_t T = (ix / r) + (int64_t)mx * ((iy / r) + (int64_t)my * (iz / r));
        double cf[3] = {cfg->lo[0] + (ix + 0.5) * hf[0], cfg->lo[1] + (iy + 0.5) * hf[1],
                        cfg->lo[2] + (iz + 0.5) * hf[2]};
        double cC[3] = {cfg->lo[0] + (ix / r + 0.5) * hc[0], cfg->lo[1] + (iy / r + 0.5) * hc[1],
                        cfg->lo[2] + (iz / r + 0.5) * hc[2]};
        for (int64_t s = cs[ci]; s < cs[ci + 1]; ++s) {
            int64_t i = perm[s];
            const double *ri = wp + 3 * i;
            double relc[3] = {ri[0] - cC[0], ri[1] - cC[1], ri[2] - cC[2]};
            double relf[3] = {ri[0] - cf[0], ri[1] - cf[1], ri[2] - cf[2]};
            double f, g[3], f2, g2[3];
            l2p(p, Lc + T * np, relc, &f, g);
            if (cfg->periodic && Qtot != 0.0) {
                double rr = relc[0] * relc[0] + relc[1] * relc[1] + relc[2] * relc[2];
                f += 2.0 * M_PI / (3.0 * V) * Qtot * (rr - 3.0 / (2.0 * cfg->alpha * cfg->alpha));
                for (int a = 0; a < 3; ++a) g[a] += 4.0 * M_PI / (3.0 * V) * Qtot * relc[a];
            }
            l2p(p, Lf + t * np, relf, &f2, g2);
            f += f2;
            for (int a = 0; a < 3; ++a) g[a] += g2[a];
            near_field(cfg, cs, perm, wp, q, i, ix, iy, iz, &f, g);
            phi[i] = f;
            for (int a = 0; a < 3; ++a) grad[3 * i + a] = g[a];
        }
    }

    free(Lf); free(Lc0); free(Lc); free(need); free(Mc); free(Mf);
    free(cell); free(perm); free(cs); free(wp);
    return 0;
}
