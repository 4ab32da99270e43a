// Zolotarev coefficients on the host, FP64 (Sec. 5.3, Eqs. Compcis, hatZ,
// ZPartialFrac2 and the l-update of Alg. 8).
//
//   c_i = l^2 sc^2(i K'/(2r+1); l'),  sc = sn/cn,  l' = sqrt(1 - l^2),  K' = K(l')
//
// evaluated with Jacobi theta series (Whittaker & Watson, ch. 21-22):
//   sn(u;k) = (th3/th2) th1(v)/th4(v),  cn(u;k) = (th4/th2) th2(v)/th4(v),
//   v = pi u / (2 K(k)),  nome q(k) = exp(-pi K(k')/K(k)),
//   th1(v) = 2 sum_{n>=0} (-1)^n q^{(n+1/2)^2} sin((2n+1)v),
//   th2(v) = 2 sum_{n>=0} q^{(n+1/2)^2} cos((2n+1)v),
//   th3(0) = 1 + 2 sum_{n>=1} q^{n^2},  th4(v) = 1 + 2 sum_{n>=1} (-1)^n q^{n^2} cos(2nv).
// Two regimes keep the nome small so the series converge in a few terms:
//   * l <= 1/sqrt2: Jacobi's imaginary transformation sc(u; l') = -i sn(iu; l)
//     turns the quantity into theta functions of the SMALL modulus l at an
//     imaginary argument (sin, cos -> sinh, cosh); with l = 1e-16 the nome is
//     ~1e-33 and sn/cn never goes through a cn near zero.
//   * l > 1/sqrt2: the modulus l' is small and sc(u; l') is taken directly
//     with the nome of l'.
// The nome comes from the series q = e + 2e^5 + 15e^9 + 150e^13 + 1707e^17,
// e = (1 - sqrt(k'))/(2(1 + sqrt(k'))) (Abramowitz & Stegun 17.3.21), with
// 1 - sqrt(k') formed without cancellation; e <= 0.0433 in both regimes.
#include <math.h>

#include "pssd_internal.h"

namespace pssd {

namespace {

// nome of the modulus k whose complementary modulus is kp (k <= 1/sqrt2)
double nome(double k, double kp)
{
    // 1 - sqrt(kp) = (1 - kp) / (1 + sqrt(kp)),  1 - kp = k^2 / (1 + kp)
    double skp = sqrt(kp);
    double one_m = (k * k / (1.0 + kp)) / (1.0 + skp);
    double e = one_m / (2.0 * (1.0 + skp));
    double e4 = e * e * e * e;
    return e * (1.0 + e4 * (2.0 + e4 * (15.0 + e4 * (150.0 + e4 * 1707.0))));
}

// l * sc(u; l') for l <= 1/sqrt2, by the imaginary transformation.
// u = t K(l') with t in [0,1).  With q = nome(l), K'/K = -ln(q)/pi and the
// theta argument is i y, y = pi u / (2 K(l)) = t (-ln q)/2.
double l_sc_small(double ell, double t)
{
    double lp = sqrt((1.0 - ell) * (1.0 + ell));
    double q = nome(ell, lp);
    double lnq = log(q);
    double y = t * (-lnq) * 0.5;
    // th2(0), th3(0)
    double th2 = 0.0, th3 = 1.0;
    for (int n = 0; n < 60; ++n) {
        double a = (n + 0.5) * (n + 0.5) * lnq;
        double t2 = 2.0 * exp(a);
        th2 += t2;
        if (n >= 1) th3 += 2.0 * exp((double)n * n * lnq);
        if (t2 < 1e-300 || a < -745.0) break;
    }
    // N = sum (-1)^n q^{(n+1/2)^2} sinh((2n+1) y),  D = 1 + 2 sum (-1)^n q^{n^2} cosh(2 n y)
    // terms written as exp(a + b) to avoid overflow of sinh / cosh
    double N = 0.0, D = 1.0;
    for (int n = 0; n < 60; ++n) {
        double a = (n + 0.5) * (n + 0.5) * lnq;
        double b = (2.0 * n + 1.0) * y;
        double term = 0.5 * (exp(a + b) - exp(a - b));
        N += (n & 1) ? -term : term;
        if (a + b < -745.0) break;
    }
    for (int n = 1; n < 60; ++n) {
        double a = (double)n * n * lnq;
        double b = 2.0 * n * y;
        double term = exp(a + b) + exp(a - b);
        D += (n & 1) ? -term : term;
        if (a + b < -745.0) break;
    }
    // l sc(u; l') = (th2/th3) * 2N / D   (l = th2^2/th3^2 and th1(iy) = 2i N)
    return (th2 / th3) * 2.0 * N / D;
}

// l * sc(u; l') for l > 1/sqrt2: modulus k = l' is small, real argument
double l_sc_large(double ell, double t)
{
    double k = sqrt((1.0 - ell) * (1.0 + ell));   // l'
    if (k == 0.0) return ell * tan(t * M_PI * 0.5);  // modulus 0: sc = tan, K = pi/2
    double q = nome(k, ell);
    double lnq = log(q);
    // v = pi u / (2 K(l')) = t pi / 2
    double v = t * M_PI * 0.5;
    double th3 = 1.0, th4 = 1.0, th1 = 0.0, th2v = 0.0;
    for (int n = 0; n < 60; ++n) {
        double a = (n + 0.5) * (n + 0.5) * lnq;
        double qa = exp(a);
        th1 += ((n & 1) ? -2.0 : 2.0) * qa * sin((2.0 * n + 1.0) * v);
        th2v += 2.0 * qa * cos((2.0 * n + 1.0) * v);
        if (n >= 1) {
            double qb = exp((double)n * n * lnq);
            th3 += 2.0 * qb;
            th4 += ((n & 1) ? -2.0 : 2.0) * qb;
        }
        if (a < -745.0) break;
    }
    // sc = sn/cn = (th3/th4) th1(v)/th2(v)
    return ell * (th3 / th4) * th1 / th2v;
}

}  // namespace

int zolo_coeffs_host(double ell, int r, double *c, double *a, double *chat, double *ell_next)
{
    if (!(ell > 0.0) || !(ell <= 1.0)) return -1;
    if (r < 1 || r > 64) return -2;
    if (!c) return -3;
    if (!a) return -4;
    if (!chat) return -5;
    if (!ell_next) return -6;
    const bool small = ell <= M_SQRT1_2;
    for (int i = 1; i <= 2 * r; ++i) {
        double t = (double)i / (2.0 * r + 1.0);
        double v = small ? l_sc_small(ell, t) : l_sc_large(ell, t);
        c[i - 1] = v * v;
    }
    for (int j = 1; j <= r; ++j) {
        double cj = c[2 * j - 2];
        double num = 1.0, den = 1.0;
        for (int k = 1; k <= r; ++k) {
            num *= cj - c[2 * k - 1];
            if (k != j) den *= cj - c[2 * k - 2];
        }
        a[j - 1] = -num / den;
    }
    double C = 1.0, prod = 1.0;
    for (int j = 1; j <= r; ++j) {
        C *= (1.0 + c[2 * j - 2]) / (1.0 + c[2 * j - 1]);
        prod *= (ell * ell + c[2 * j - 1]) / (ell * ell + c[2 * j - 2]);
    }
    *chat = C;
    *ell_next = C * ell * prod;
    return 0;
}

int choose_r_host(double ell, double tau, int r_max)
{
    double c[128], a[64], ch, l1, l2;
    if (r_max > 64) r_max = 64;
    for (int r = 1; r <= r_max; ++r) {
        if (zolo_coeffs_host(ell, r, c, a, &ch, &l1)) return r_max;
        if (l1 > 1.0) l1 = 1.0;
        if (1.0 - l1 <= tau) return r;
        if (zolo_coeffs_host(l1, r, c, a, &ch, &l2)) return r_max;
        if (1.0 - l2 <= tau) return r;
    }
    return r_max;
}

}  // namespace pssd
