// An operation-counting scalar.  TEST INFRASTRUCTURE: compiling the oracle's
// own arithmetic with it (oracle/volna_oracle_count.cpp) counts the
// floating-point operations the scheme performs on state-dependent values per
// step -- the algorithmic flop count used for the FP64 roofline.  Geometry
// (plain double) is precomputed and not counted.  Single-threaded.
#pragma once

#include <cmath>
#include <cstdint>

struct VoOpCounts {
    int64_t add = 0, sub = 0, mul = 0, div = 0, sqrt = 0, minmax = 0;
};

inline VoOpCounts &vo_counts()
{
    static VoOpCounts c;
    return c;
}

struct cdouble {
    double v;
    cdouble() = default;
    cdouble(double x) : v(x) {}
};

inline cdouble operator+(cdouble a, cdouble b) { vo_counts().add++; return cdouble(a.v + b.v); }
inline cdouble operator-(cdouble a, cdouble b) { vo_counts().sub++; return cdouble(a.v - b.v); }
inline cdouble operator*(cdouble a, cdouble b) { vo_counts().mul++; return cdouble(a.v * b.v); }
inline cdouble operator/(cdouble a, cdouble b) { vo_counts().div++; return cdouble(a.v / b.v); }
inline cdouble operator-(cdouble a) { return cdouble(-a.v); }
inline cdouble &operator+=(cdouble &a, cdouble b) { return a = a + b; }

inline bool operator<(cdouble a, cdouble b) { return a.v < b.v; }
inline bool operator>(cdouble a, cdouble b) { return a.v > b.v; }
inline bool operator<=(cdouble a, cdouble b) { return a.v <= b.v; }
inline bool operator>=(cdouble a, cdouble b) { return a.v >= b.v; }
inline bool operator==(cdouble a, cdouble b) { return a.v == b.v; }
inline bool operator!=(cdouble a, cdouble b) { return a.v != b.v; }

inline cdouble sqrt(cdouble a) { vo_counts().sqrt++; return cdouble(std::sqrt(a.v)); }
inline cdouble fabs(cdouble a) { vo_counts().minmax++; return cdouble(std::fabs(a.v)); }
inline cdouble fmin(cdouble a, cdouble b) { vo_counts().minmax++; return b.v < a.v ? b : a; }
inline cdouble fmax(cdouble a, cdouble b) { vo_counts().minmax++; return b.v > a.v ? b : a; }
