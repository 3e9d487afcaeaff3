// flop_count.cpp -- counts the floating-point operations of one step of the
// oracle (oracle.c, unchanged) by compiling it as C++ with `double` replaced by
// a value type whose +, -, *, / and sqrt (and exp, log, pow) increment
// counters.  min, max, abs, sign copies, comparisons and negation are not
// counted.  The counts are the algorithmic work per cell update that the
// benchmark divides by a kernel's time for its ALU roofline.
//
// TEST AND MEASUREMENT INFRASTRUCTURE, like the rest of oracle/: only the
// tests read its output (the benchmark's FLOP constants are pinned to it).
//
// usage: flop_count <workload> <n>
//   sw2d       classic 2D shallow water, Roe + Harten-Hyman, MC, transverse 2,
//              one step on an n x n grid of smooth data with every wave
//              non-zero and no transonic rarefaction
//   euler2d    SharpClaw 2D Euler, WENO5 characteristic-wise: one evaluation
//              of L(Q) (one SSP stage) on an n x n grid of smooth data
//   elast1d    classic 1D nonlinear elasticity, f-waves, MC: one step on n
//              cells of a layered medium
//   acou1d     classic 1D linear acoustics (rho = 1, K = 4), MC: one step on
//              n periodic cells of smooth data
// prints one JSON object: operations per cell by kind, the total, and the
// operations of one Roe-average evaluation (sw2d, euler2d).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <cmath>

namespace {
long long n_add = 0, n_mul = 0, n_div = 0, n_sqrt = 0, n_tr = 0;
}

// a double that counts the arithmetic done on it
struct CD {
  double v;
  CD() : v(0) {}
  CD(double x) : v(x) {}
  CD(int x) : v(x) {}
  CD(long x) : v((double)x) {}
  CD(long long x) : v((double)x) {}
  CD(unsigned x) : v(x) {}
  CD(unsigned long x) : v((double)x) {}
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned long() const { return (unsigned long)v; }
  explicit operator bool() const { return v != 0; }
  CD& operator+=(CD o) { ++n_add; v += o.v; return *this; }
  CD& operator-=(CD o) { ++n_add; v -= o.v; return *this; }
  CD& operator*=(CD o) { ++n_mul; v *= o.v; return *this; }
  CD& operator/=(CD o) { ++n_div; v /= o.v; return *this; }
  CD operator-() const { return CD(-v); }
  CD operator+() const { return *this; }
};
inline CD operator+(CD a, CD b) { ++n_add; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++n_add; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++n_mul; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++n_div; return CD(a.v / b.v); }
inline bool operator<(CD a, CD b) { return a.v < b.v; }
inline bool operator>(CD a, CD b) { return a.v > b.v; }
inline bool operator<=(CD a, CD b) { return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { return a.v >= b.v; }
inline bool operator==(CD a, CD b) { return a.v == b.v; }
inline bool operator!=(CD a, CD b) { return a.v != b.v; }
inline CD sqrt(CD a) { ++n_sqrt; return CD(std::sqrt(a.v)); }
inline CD exp(CD a) { ++n_tr; return CD(std::exp(a.v)); }
inline CD log(CD a) { ++n_tr; return CD(std::log(a.v)); }
inline CD log1p(CD a) { ++n_tr; return CD(std::log1p(a.v)); }
inline CD pow(CD a, CD b) { ++n_tr; return CD(std::pow(a.v, b.v)); }
inline CD fma(CD a, CD b, CD c) {
  ++n_mul;
  ++n_add;
  return CD(std::fma(a.v, b.v, c.v));
}
inline CD fabs(CD a) { return CD(std::fabs(a.v)); }
inline CD fmin(CD a, CD b) { return CD(std::fmin(a.v, b.v)); }
inline CD fmax(CD a, CD b) { return CD(std::fmax(a.v, b.v)); }
inline CD copysign(CD a, CD b) { return CD(std::copysign(a.v, b.v)); }
inline CD floor(CD a) { return CD(std::floor(a.v)); }
inline bool isnan(CD a) { return std::isnan(a.v); }
inline bool isfinite(CD a) { return std::isfinite(a.v); }
inline bool isinf(CD a) { return std::isinf(a.v); }

#define double CD
#include "oracle.c"
#undef double

namespace {

void reset() { n_add = n_mul = n_div = n_sqrt = n_tr = 0; }
long long total() { return n_add + n_mul + n_div + n_sqrt + n_tr; }

void base(orc_prob& P, int ndim, int nx, int ny, int rp, int m, int nw) {
  memset(&P, 0, sizeof(P));
  P.ndim = ndim;
  P.nx = nx;
  P.ny = ny;
  P.nz = 1;
  P.dx = 1.0 / nx;
  P.dy = 1.0 / ny;
  P.dz = 1.0;
  P.rp = rp;
  P.lim = ORC_LIM_MC;
  P.order = 2;
  P.transverse = ndim == 2 ? 2 : 0;
  P.entropy_fix = 1;
  P.num_eqn = m;
  P.num_waves = nw;
  P.capa_index = -1;
  for (int d = 0; d < 3; ++d) P.bc_lo[d] = P.bc_hi[d] = ORC_BC_PERIODIC;
  P.cfl_desired = 0.9;
  P.cfl_max = 1.0;
  P.dt_max = 1e30;
  P.max_retries = 8;
  P.weno_eps = 1e-6;
}

void report(const char* w, long long cells, long long roe) {
  printf("{\"workload\": \"%s\", \"cells\": %lld, \"add\": %.4f, \"mul\": %.4f, \"div\": %.4f, "
         "\"sqrt\": %.4f, \"transcendental\": %.4f, \"total\": %.4f, \"roe_average\": %lld}\n",
         w, cells, (double)n_add / cells, (double)n_mul / cells, (double)n_div / cells,
         (double)n_sqrt / cells, (double)n_tr / cells, (double)total() / cells, roe);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 3) {
    fprintf(stderr, "usage: flop_count sw2d|euler2d|elast1d|acou1d n\n");
    return 2;
  }
  const char* w = argv[1];
  const int n = atoi(argv[2]);
  orc_prob P;
  if (!strcmp(w, "sw2d")) {
    base(P, 2, n, n, ORC_RP_SW_ROE, 3, 3);
    P.params[0] = 1.0;
    CD* q = (CD*)malloc(sizeof(CD) * 3 * n * n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const double x = (i + 0.5) / n, y = (j + 0.5) / n, tp = 2 * M_PI;
        q[j * n + i] = 1.5 + 0.2 * std::sin(tp * x) * std::cos(tp * y);
        q[n * n + j * n + i] = 0.3 * std::sin(tp * (x - y)) + 0.05;
        q[2 * n * n + j * n + i] = 0.2 * std::cos(tp * (x + 2 * y)) + 0.05;
      }
    // one Roe average (the transverse solver re-derives it per call)
    CD ql[3] = {q[0], q[n * n], q[2 * n * n]}, qr[3] = {q[1], q[n * n + 1], q[2 * n * n + 1]};
    CD un, ut, c;
    reset();
    sw_roe_avg(&P, 0, ql, qr, &un, &ut, &c);
    const long long roe = total();
    CD cfl;
    reset();
    orc_classic_step(&P, q, nullptr, CD(0.2 / n), &cfl);
    report(w, (long long)n * n, roe);
    free(q);
  } else if (!strcmp(w, "euler2d")) {
    base(P, 2, n, n, ORC_RP_EULER_ROE, 4, 4);
    P.scheme = ORC_SHARPCLAW;
    P.char_decomp = 1;
    P.weno_r = 3;
    P.params[0] = 1.4;
    CD* q = (CD*)malloc(sizeof(CD) * 4 * n * n);
    CD* L = (CD*)malloc(sizeof(CD) * 4 * n * n);
    const long long c2 = (long long)n * n;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const double x = (i + 0.5) / n, y = (j + 0.5) / n, tp = 2 * M_PI;
        const double rho = 1.5 + 0.2 * std::sin(tp * x) * std::cos(tp * y);
        const double u = 0.3 * std::sin(tp * (x - y)) + 0.05;
        const double v = 0.2 * std::cos(tp * (x + 2 * y)) + 0.05;
        const double p = 1.5 + 0.2 * std::cos(tp * (2 * x + y));
        q[j * n + i] = rho;
        q[c2 + j * n + i] = rho * u;
        q[2 * c2 + j * n + i] = rho * v;
        q[3 * c2 + j * n + i] = p / 0.4 + 0.5 * rho * (u * u + v * v);
      }
    CD ql[4] = {q[0], q[c2], q[2 * c2], q[3 * c2]};
    CD qr[4] = {q[1], q[c2 + 1], q[2 * c2 + 1], q[3 * c2 + 1]};
    CD un, ut, H, c, cc;
    reset();
    euler_roe_avg(&P, 0, ql, qr, &un, &ut, &H, &c, &cc);
    const long long roe = total();
    CD smax[2];
    reset();
    orc_sharp_L(&P, q, nullptr, L, smax);
    report(w, c2, roe);
    free(q);
    free(L);
  } else if (!strcmp(w, "elast1d")) {
    base(P, 1, n, 1, ORC_RP_ELASTICITY_FWAVE, 2, 2);
    P.num_aux = 2;
    CD* q = (CD*)malloc(sizeof(CD) * 2 * n);
    CD* aux = (CD*)malloc(sizeof(CD) * 2 * n);
    for (int i = 0; i < n; ++i) {
      const double x = (i + 0.5) / n;
      const int layer = ((int)(x * 16)) & 1;
      aux[i] = layer ? 4.0 : 1.0;
      aux[n + i] = layer ? 4.0 : 1.0;
      q[i] = 0.05 * std::sin(2 * M_PI * x) + 0.01;
      q[n + i] = 0.1 * std::cos(2 * M_PI * x) + 0.01;
    }
    CD cfl;
    reset();
    orc_classic_step(&P, q, aux, CD(0.2 / n), &cfl);
    report(w, n, 0);
    free(q);
    free(aux);
  } else if (!strcmp(w, "acou1d")) {
    base(P, 1, n, 1, ORC_RP_ACOUSTICS, 2, 2);
    P.params[0] = 1.0;
    P.params[1] = 4.0;
    CD* q = (CD*)malloc(sizeof(CD) * 2 * n);
    for (int i = 0; i < n; ++i) {
      const double x = (i + 0.5) / n;
      q[i] = 1.0 + 0.5 * std::sin(2 * M_PI * x);
      q[n + i] = 0.25 * std::cos(2 * M_PI * x);
    }
    CD cfl;
    reset();
    orc_classic_step(&P, q, nullptr, CD(0.2 / n), &cfl);
    report(w, n, 0);
    free(q);
  } else {
    fprintf(stderr, "unknown workload %s\n", w);
    return 2;
  }
  return 0;
}
