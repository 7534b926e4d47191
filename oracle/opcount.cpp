// Op-counting build of the oracle (measurement infrastructure, never on the
// product path).  The oracle source is compiled as C++ with `real` a double
// that counts every FP64 operation with at least one operand derived from the
// state; operations on constants only (folded by any compiler) are not
// counted.  Each of + - * / sqrt pow counts one algorithmic flop; negation,
// fabs and comparisons count none.
#include <cmath>

namespace opc {
long long add = 0, mul = 0, dvd = 0, sqr = 0, pw = 0;
int phase = 0, saved_phase = 0;
long long by_phase[4][5];
long long n_equal = 0;
}

struct real {
  double v;
  bool k;   // known constant (not derived from the state)
  real() : v(0.0), k(true) {}
  real(double x) : v(x), k(true) {}
  operator double() const { return v; }
};

static inline real mk(double v, bool k) { real r(v); r.k = k; return r; }
static inline void set_phase(int k)
{
  long long now[5] = {opc::add, opc::mul, opc::dvd, opc::sqr, opc::pw};
  static long long last[5];
  for (int i = 0; i < 5; ++i) { opc::by_phase[opc::phase][i] += now[i] - last[i]; last[i] = now[i]; }
  opc::phase = k;
}
static inline real or_data(double x) { return mk(x, false); }

// Leading Riemann problems whose traces agree to within 2^-48 (each
// component relative to the sum of its two values, the momentum on the
// sqrt(rho E) scale) have equal data: their exact solution is the constant
// state.  Their operations go to bucket 3, so the count of the method that
// resolves equal data without iterating is the flux bucket plus the cost of
// the test.  Counting only: no value changes.
static inline void leading_rp(const real *L, const real *R, int k)
{
  if (k == 0) {
    const double e = 3.552713678800501e-15;
    const double sr = L[0].v + R[0].v, sE = L[2].v + R[2].v, dm = R[1].v - L[1].v;
    if (std::fabs(R[0].v - L[0].v) <= e * sr && std::fabs(R[2].v - L[2].v) <= e * sE && dm * dm <= e * e * sr * sE) {
      ++opc::n_equal;
      opc::saved_phase = opc::phase;
      set_phase(3);
    }
  } else if (opc::phase == 3) {
    set_phase(opc::saved_phase);
  }
}

#define OR_REAL_DEFINED
#define OR_DATA(x) or_data(x)
#define OR_PHASE(k) set_phase(k)
#define OR_LEADING_RP(L, R, k) leading_rp(L, R, k)

#define BINOP(OP, CTR)                                                                               \
  static inline real operator OP(real a, real b) { if (!(a.k && b.k)) ++opc::CTR; return mk(a.v OP b.v, a.k && b.k); } \
  static inline real operator OP(real a, double b) { return a OP real(b); }                         \
  static inline real operator OP(double a, real b) { return real(a) OP b; }                         \
  static inline real operator OP(real a, int b) { return a OP real((double)b); }                    \
  static inline real operator OP(int a, real b) { return real((double)a) OP b; }
BINOP(+, add)
BINOP(-, add)
BINOP(*, mul)
BINOP(/, dvd)
#define CMPOP(OP)                                                                  \
  static inline bool operator OP(real a, real b) { return a.v OP b.v; }            \
  static inline bool operator OP(real a, double b) { return a.v OP b; }            \
  static inline bool operator OP(double a, real b) { return a OP b.v; }            \
  static inline bool operator OP(real a, int b) { return a.v OP (double)b; }       \
  static inline bool operator OP(int a, real b) { return (double)a OP b.v; }
CMPOP(<)
CMPOP(>)
CMPOP(<=)
CMPOP(>=)
CMPOP(==)
CMPOP(!=)
static inline real operator-(real a) { return mk(-a.v, a.k); }
static inline bool operator!(real a) { return !a.v; }
static inline real sqrt(real a) { if (!a.k) ++opc::sqr; return mk(std::sqrt(a.v), a.k); }
static inline real fabs(real a) { return mk(std::fabs(a.v), a.k); }
static inline real pow(real a, real b) { if (!(a.k && b.k)) ++opc::pw; return mk(std::pow(a.v, b.v), a.k && b.k); }
static inline real pow(real a, double b) { return pow(a, real(b)); }

#include "grprec_oracle.c"

// out[phase * 5 + kind]: phases CFL, reconstruction + GRP, update + repair,
// leading Riemann problems with equal data; kinds add, mul, div, sqrt, pow;
// out[20]: the number of those Riemann problems (a single-threaded run is
// assumed)
extern "C" void or_opcount(long long *out)
{
  set_phase(opc::phase);
  for (int p = 0; p < 4; ++p)
    for (int i = 0; i < 5; ++i) out[p * 5 + i] = opc::by_phase[p][i];
  out[20] = opc::n_equal;
}

extern "C" void or_opcount_reset(void)
{
  set_phase(0);
  for (int p = 0; p < 4; ++p)
    for (int i = 0; i < 5; ++i) opc::by_phase[p][i] = 0;
  opc::n_equal = 0;
}
