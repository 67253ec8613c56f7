// A minimal reverse-mode (tape) automatic-differentiation scalar.  TEST
// INFRASTRUCTURE: it turns the oracle's own arithmetic into the oracle's
// discrete adjoint (oracle/volna_oracle_ad.cpp), so the hand-written GPU adjoint
// is checked against the derivative of an independent program.
//
// Every operation on an active value appends one node to a global tape: the
// indices of (at most) two operands and the partial derivatives with respect to
// them.  The reverse sweep walks the tape backwards.  Branching functions
// (min, max, fabs, comparisons) follow the branch taken by the values, with
// ties resolved towards the first argument.  Single-threaded.
#pragma once

#include <cmath>
#include <cstdint>
#include <vector>

struct VoTape {
    std::vector<int32_t> a0, a1;
    std::vector<double> d0, d1;
    void clear()
    {
        a0.clear(); a1.clear(); d0.clear(); d1.clear();
    }
    int32_t push(int32_t i0, double p0, int32_t i1, double p1)
    {
        a0.push_back(i0); d0.push_back(p0);
        a1.push_back(i1); d1.push_back(p1);
        return (int32_t)(a0.size() - 1);
    }
    size_t size() const { return a0.size(); }
    // adj has size() entries; seeds set by the caller; propagates to operands.
    void reverse(std::vector<double> &adj) const
    {
        for (size_t k = a0.size(); k-- > 0;) {
            double g = adj[k];
            if (g == 0.0) continue;
            if (a0[k] >= 0) adj[a0[k]] += d0[k] * g;
            if (a1[k] >= 0) adj[a1[k]] += d1[k] * g;
        }
    }
};

inline VoTape &vo_tape()
{
    static VoTape t;
    return t;
}

struct adouble {
    double v;
    int32_t i;    // tape node, -1 for a constant
    adouble() = default;
    adouble(double x) : v(x), i(-1) {}
    static adouble variable(double x)
    {
        adouble r;
        r.v = x;
        r.i = vo_tape().push(-1, 0.0, -1, 0.0);
        return r;
    }
};

inline adouble ad_node(double v, int32_t i0, double p0, int32_t i1, double p1)
{
    adouble r;
    r.v = v;
    if (i0 < 0 && i1 < 0) {
        r.i = -1;
        return r;
    }
    r.i = vo_tape().push(i0, p0, i1, p1);
    return r;
}

inline adouble operator+(adouble a, adouble b) { return ad_node(a.v + b.v, a.i, 1.0, b.i, 1.0); }
inline adouble operator-(adouble a, adouble b) { return ad_node(a.v - b.v, a.i, 1.0, b.i, -1.0); }
inline adouble operator*(adouble a, adouble b) { return ad_node(a.v * b.v, a.i, b.v, b.i, a.v); }
inline adouble operator/(adouble a, adouble b)
{
    double r = a.v / b.v;
    return ad_node(r, a.i, 1.0 / b.v, b.i, -r / b.v);
}
inline adouble operator-(adouble a) { return ad_node(-a.v, a.i, -1.0, -1, 0.0); }
inline adouble &operator+=(adouble &a, adouble b) { return a = a + b; }

inline bool operator<(adouble a, adouble b) { return a.v < b.v; }
inline bool operator>(adouble a, adouble b) { return a.v > b.v; }
inline bool operator<=(adouble a, adouble b) { return a.v <= b.v; }
inline bool operator>=(adouble a, adouble b) { return a.v >= b.v; }
inline bool operator==(adouble a, adouble b) { return a.v == b.v; }
inline bool operator!=(adouble a, adouble b) { return a.v != b.v; }

inline adouble sqrt(adouble a)
{
    double r = std::sqrt(a.v);
    return ad_node(r, a.i, r > 0.0 ? 0.5 / r : 0.0, -1, 0.0);
}
inline adouble fabs(adouble a) { return a.v < 0.0 ? -a : a; }
inline adouble fmin(adouble a, adouble b) { return b.v < a.v ? b : a; }
inline adouble fmax(adouble a, adouble b) { return b.v > a.v ? b : a; }
