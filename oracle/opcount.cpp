/*
 * opcount.cpp -- floating-point operation counter of the oracle's inversion.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY (see orc.h).  The oracle's own
 * physics.c and con2prim.c (Sections 2.1 and 2.3) are compiled a second time
 * here, unchanged, with every `double` replaced by the counting scalar Num:
 * each arithmetic operation on a Num adds to a tally by kind.  The tally is
 * the method's algorithmic FP64 work as the plain oracle performs it (no
 * fused multiply-adds, one operation per source-level +, -, *, /), the
 * numerator of the FP64-peak fraction of an inversion.
 *
 * Counted: add/sub, mul, div, sqrt (one flop each), and calls of pow / exp /
 * log (reported apart, not in the flop total); comparisons, fabs, negation,
 * copies and conversions are not arithmetic and are not counted.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <cmath>

namespace orc_count {

struct Tally {
    long long add, mul, div, sqrt, special;
};
static thread_local Tally T;

struct Num {
    double v;
    Num() : v(0.0) {}
    Num(double x) : v(x) {}
    Num(int x) : v((double)x) {}
    Num(long x) : v((double)x) {}
    explicit operator int() const { return (int)v; }
};

inline Num operator+(Num a, Num b) { T.add++; return Num(a.v + b.v); }
inline Num operator-(Num a, Num b) { T.add++; return Num(a.v - b.v); }
inline Num operator*(Num a, Num b) { T.mul++; return Num(a.v * b.v); }
inline Num operator/(Num a, Num b) { T.div++; return Num(a.v / b.v); }
inline Num operator-(Num a) { return Num(-a.v); }
inline Num operator+(Num a) { return a; }
inline Num &operator+=(Num &a, Num b) { a = a + b; return a; }
inline Num &operator-=(Num &a, Num b) { a = a - b; return a; }
inline Num &operator*=(Num &a, Num b) { a = a * b; return a; }
inline Num &operator/=(Num &a, Num b) { a = a / b; return a; }
inline bool operator<(Num a, Num b) { return a.v < b.v; }
inline bool operator>(Num a, Num b) { return a.v > b.v; }
inline bool operator<=(Num a, Num b) { return a.v <= b.v; }
inline bool operator>=(Num a, Num b) { return a.v >= b.v; }
inline bool operator==(Num a, Num b) { return a.v == b.v; }
inline bool operator!=(Num a, Num b) { return a.v != b.v; }
inline Num sqrt(Num a) { T.sqrt++; return Num(std::sqrt(a.v)); }
inline Num fabs(Num a) { return Num(std::fabs(a.v)); }
inline Num pow(Num a, Num b) { T.special++; return Num(std::pow(a.v, b.v)); }
inline Num exp(Num a) { T.special++; return Num(std::exp(a.v)); }
inline Num log(Num a) { T.special++; return Num(std::log(a.v)); }
inline Num fmin(Num a, Num b) { return Num(std::fmin(a.v, b.v)); }
inline Num fmax(Num a, Num b) { return Num(std::fmax(a.v, b.v)); }
inline bool isfinite(Num a) { return std::isfinite(a.v); }

#define double Num
#include "orc.h"
#include "physics.c"
#include "con2prim.c"
#undef double

} // namespace orc_count

/* Inversion of one state by the oracle's con2prim, counted.  geom34: gcov
 * (16), gcon (16), sqrt(-g), alpha of the point; gam, nr_tol, beta_entropy,
 * nr_maxit, brent_maxit: the solver parameters (Sections 2.3-2.4); wguess > 0:
 * Newton first starts from that W (orc_con2prim_w); out[0..5] = add, mul,
 * div, sqrt, pow/exp/log calls, flops (the first four summed); P, the
 * returned flag and iters as the oracle's inversion gives them. */
extern "C" int orc_count_con2prim(const double *U, const double *geom34, const double *guess, double gam,
                                  double nr_tol, double beta_entropy, int nr_maxit, int brent_maxit,
                                  int methods, double wguess, double *P, int *iters, long long *out)
{
    using namespace orc_count;
    orc_params pn;
    memset((void *)&pn, 0, sizeof(pn));
    pn.gam = gam;
    pn.nr_tol = nr_tol;
    pn.beta_entropy = beta_entropy;
    pn.nr_maxit = nr_maxit;
    pn.brent_maxit = brent_maxit;
    orc_geom g;
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            g.gcov[m][n] = geom34[4 * m + n];
            g.gcon[m][n] = geom34[16 + 4 * m + n];
        }
    g.gdet = geom34[32];
    g.alpha = geom34[33];
    Num Un[ORC_NU], gn[ORC_NP], Pn[ORC_NP];
    for (int c = 0; c < ORC_NU; c++) Un[c] = U[c];
    for (int c = 0; c < ORC_NP; c++) gn[c] = guess[c];
    T = Tally{0, 0, 0, 0, 0};
    int fl = orc_con2prim_w(Un, &g, gn, &pn, Pn, iters, methods, Num(wguess));
    Tally t = T;
    for (int c = 0; c < ORC_NP; c++) P[c] = Pn[c].v;
    out[0] = t.add; out[1] = t.mul; out[2] = t.div; out[3] = t.sqrt; out[4] = t.special;
    out[5] = t.add + t.mul + t.div + t.sqrt;
    return fl;
}
