// opcount.cpp -- operation counts of the CPU oracle (test infrastructure).
//
// The oracle source afns_oracle.c is compiled here a second time, as C++, with
// every `double` replaced by a counting scalar: each arithmetic operation the
// oracle performs is tallied by kind (add/subtract, multiply, divide, square
// root, exponential/trigonometric/logarithm, and the non-arithmetic compares,
// min/max, |x| and negations), by step of the stage (the ORC_PHASE marks in the
// oracle) and by how it arises:
//   counted   -- a nontrivial operation in the first evaluation of a quantity;
//   repeated  -- an operation inside a pure function (ORC_PURE marks) that was
//                already evaluated with the same inputs during this residual
//                (the oracle re-evaluates shared node quantities per use);
//   trivial   -- an add/subtract with an exact zero operand or a multiply with
//                an exact 0 or +-1 operand (the zero entries of the K matrices,
//                the zero coefficients of the full Runge-Kutta table).
// The values the oracle computes are the plain doubles inside the counting type,
// so the arithmetic is the oracle's own; nothing here changes it. Loaded only by
// the tests and by bench.py's measurement of the algorithmic work per cell.
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

namespace cnt {

enum { ADD = 0, MUL, DIV, SQRT, TRANS, OTHER, NCAT };
enum { COUNTED = 0, REPEATED, TRIVIAL, NKIND };
constexpr int NPH = 12;

static long long tally[NPH][NCAT][NKIND];
static int phase = 0;
static int repeat_depth = 0;
static std::unordered_set<std::string> seen;

inline void op(int cat, bool trivial = false)
{
    const int kind = repeat_depth > 0 ? REPEATED : trivial ? TRIVIAL : COUNTED;
    ++tally[phase][cat][kind];
}

inline void set_phase(int k)
{
    // phase 0 opens a residual evaluation: pure evaluations start afresh
    if (k == 0) seen.clear();
    phase = k;
}

struct Real {
    double v;
    Real() = default;
    Real(double x) : v(x) {}
    explicit operator double() const { return v; }
    Real &operator+=(Real b);
    Real &operator-=(Real b);
    Real &operator*=(Real b);
    Real &operator/=(Real b);
};

inline bool is_one(double x) { return x == 1.0 || x == -1.0; }

inline Real operator+(Real a, Real b) { op(ADD, a.v == 0.0 || b.v == 0.0); return Real(a.v + b.v); }
inline Real operator-(Real a, Real b) { op(ADD, a.v == 0.0 || b.v == 0.0); return Real(a.v - b.v); }
inline Real operator*(Real a, Real b)
{
    op(MUL, a.v == 0.0 || b.v == 0.0 || is_one(a.v) || is_one(b.v));
    return Real(a.v * b.v);
}
inline Real operator/(Real a, Real b) { op(DIV, is_one(b.v)); return Real(a.v / b.v); }
inline Real operator-(Real a) { op(OTHER); return Real(-a.v); }
inline Real operator+(Real a) { return a; }
inline Real &Real::operator+=(Real b) { return *this = *this + b; }
inline Real &Real::operator-=(Real b) { return *this = *this - b; }
inline Real &Real::operator*=(Real b) { return *this = *this * b; }
inline Real &Real::operator/=(Real b) { return *this = *this / b; }
inline bool operator<(Real a, Real b) { op(OTHER); return a.v < b.v; }
inline bool operator>(Real a, Real b) { op(OTHER); return a.v > b.v; }
inline bool operator<=(Real a, Real b) { op(OTHER); return a.v <= b.v; }
inline bool operator>=(Real a, Real b) { op(OTHER); return a.v >= b.v; }
inline bool operator==(Real a, Real b) { op(OTHER); return a.v == b.v; }
inline bool operator!=(Real a, Real b) { op(OTHER); return a.v != b.v; }

// The rest of a pure function: counted as a repeat when its inputs were seen.
struct Pure {
    bool rep;
    template <class A, class B>
    Pure(int id, const A *a, int na, const B *b, int nb, int i, int j)
    {
        std::string key(reinterpret_cast<const char *>(&id), sizeof id);
        key.append(reinterpret_cast<const char *>(&i), sizeof i);
        key.append(reinterpret_cast<const char *>(&j), sizeof j);
        if (a) key.append(reinterpret_cast<const char *>(a), sizeof(A) * (size_t)na);
        key.push_back('|');
        if (b) key.append(reinterpret_cast<const char *>(b), sizeof(B) * (size_t)nb);
        rep = !seen.insert(key).second;
        if (rep) ++repeat_depth;
    }
    ~Pure()
    {
        if (rep) --repeat_depth;
    }
};

}  // namespace cnt

using cnt::Real;

inline Real sqrt(Real a) { cnt::op(cnt::SQRT); return Real(std::sqrt(a.v)); }
inline Real exp(Real a) { cnt::op(cnt::TRANS); return Real(std::exp(a.v)); }
inline Real log(Real a) { cnt::op(cnt::TRANS); return Real(std::log(a.v)); }
inline Real sin(Real a) { cnt::op(cnt::TRANS); return Real(std::sin(a.v)); }
inline Real cos(Real a) { cnt::op(cnt::TRANS); return Real(std::cos(a.v)); }
inline Real fabs(Real a) { cnt::op(cnt::OTHER); return Real(std::fabs(a.v)); }
inline Real fmin(Real a, Real b) { cnt::op(cnt::OTHER); return Real(std::fmin(a.v, b.v)); }
inline Real fmax(Real a, Real b) { cnt::op(cnt::OTHER); return Real(std::fmax(a.v, b.v)); }
inline bool isfinite(Real a) { return std::isfinite(a.v); }

#define ORC_PHASE(k) (cnt::set_phase(k))
#define ORC_PURE(id, a, na, b, nb, i, j) cnt::Pure orc_pure_scope_((id), (a), (na), (b), (nb), (i), (j))
#define double Real
extern "C" {
#include "afns_oracle.c"
}
#undef double

extern "C" {

// Tallies [phase][category][kind] of everything since the last reset.
void orc_opcount_reset(void)
{
    std::memset(cnt::tally, 0, sizeof cnt::tally);
    cnt::seen.clear();
    cnt::phase = 0;
}

void orc_opcount_get(long long *out)
{
    std::memcpy(out, cnt::tally, sizeof cnt::tally);
}

// Counts one limited stage residual (orc_residual) of the given state; the
// residual itself is written to L_out (may be null).
int orc_opcount_residual(const orc_problem *P, const double *state, double dt, double *L_out)
{
    const size_t n = orc_state_len(P);
    std::vector<Real> s(state, state + n), L(n);
    int nb = 0;
    const int rc = orc_residual(P, s.data(), Real(dt), L.data(), nullptr, nullptr, &nb);
    if (L_out)
        for (size_t k = 0; k < n; ++k) L_out[k] = L[k].v;
    return rc;
}

// Counts one SSP-RK54 step (five residuals, the combinations, wall fixes).
int orc_opcount_step(const orc_problem *P, double *state, double dt)
{
    const size_t n = orc_state_len(P);
    std::vector<Real> s(state, state + n);
    Real taken(0.0);
    int h = 0;
    const int rc = orc_step(P, s.data(), Real(dt), 0, &taken, &h);
    for (size_t k = 0; k < n; ++k) state[k] = s[k].v;
    return rc;
}

// Counts the CFL bound of Eq. (13) (phase 9).
double orc_opcount_dt_max(const orc_problem *P, const double *state)
{
    const size_t n = orc_state_len(P);
    std::vector<Real> s(state, state + n);
    cnt::set_phase(9);
    return orc_dt_max(P, s.data()).v;
}

}  // extern "C"
