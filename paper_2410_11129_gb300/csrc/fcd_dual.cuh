// fcd_dual.cuh -- forward-mode dual numbers for the tangent-linear step.
//
// Dual<K> carries a value and its derivatives along K directions of the
// parameter space; every operation applies the chain rule to all K at once.
// Comparisons look at the value only, so branches (clamps, thresholds) take
// the primal path and differentiate the branch that was taken.
#pragma once

#include <cmath>

namespace fcd {

using ::sqrt;  // the float and double overloads stay visible next to the dual one

template <int K>
struct Dual {
    double v;
    double d[K];

    Dual() = default;  // trivial, so that dual tiles can live in shared memory
    __host__ __device__ constexpr Dual(double x) : v(x), d{} {}  // a constant
    __host__ __device__ constexpr Dual(int x) : v(double(x)), d{} {}

    __host__ __device__ Dual &operator+=(const Dual &b) {
#pragma unroll
        for (int i = 0; i < K; i++) d[i] += b.d[i];
        v += b.v;
        return *this;
    }
    __host__ __device__ Dual &operator-=(const Dual &b) {
#pragma unroll
        for (int i = 0; i < K; i++) d[i] -= b.d[i];
        v -= b.v;
        return *this;
    }
    __host__ __device__ Dual &operator+=(double b) {
        v += b;
        return *this;
    }
    __host__ __device__ Dual &operator-=(double b) {
        v -= b;
        return *this;
    }
};

template <int K>
__host__ __device__ inline Dual<K> operator-(const Dual<K> &a) {
    Dual<K> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = -a.d[i];
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator+(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator-(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator*(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator/(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    const double ib = 1.0 / b.v;
    r.v = a.v / b.v;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
// mixed with plain constants (no derivative work for the constant)
template <int K>
__host__ __device__ inline Dual<K> operator+(const Dual<K> &a, double b) {
    Dual<K> r = a;
    r.v = a.v + b;
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator+(double a, const Dual<K> &b) {
    Dual<K> r = b;
    r.v = a + b.v;
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator-(const Dual<K> &a, double b) {
    Dual<K> r = a;
    r.v = a.v - b;
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator-(double a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a - b.v;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = -b.d[i];
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator*(const Dual<K> &a, double b) {
    Dual<K> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.d[i] * b;
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator*(double a, const Dual<K> &b) {
    return b * a;
}
template <int K>
__host__ __device__ inline Dual<K> operator/(const Dual<K> &a, double b) {
    Dual<K> r;
    r.v = a.v / b;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.d[i] / b;
    return r;
}
template <int K>
__host__ __device__ inline Dual<K> operator/(double a, const Dual<K> &b) {
    return Dual<K>(a) / b;
}

// comparisons on the value
template <int K>
__host__ __device__ inline bool operator<(const Dual<K> &a, const Dual<K> &b) { return a.v < b.v; }
template <int K>
__host__ __device__ inline bool operator>(const Dual<K> &a, const Dual<K> &b) { return a.v > b.v; }
template <int K>
__host__ __device__ inline bool operator<=(const Dual<K> &a, const Dual<K> &b) { return a.v <= b.v; }
template <int K>
__host__ __device__ inline bool operator>=(const Dual<K> &a, const Dual<K> &b) { return a.v >= b.v; }
template <int K>
__host__ __device__ inline bool operator<(const Dual<K> &a, double b) { return a.v < b; }
template <int K>
__host__ __device__ inline bool operator>(const Dual<K> &a, double b) { return a.v > b; }
template <int K>
__host__ __device__ inline bool operator<=(const Dual<K> &a, double b) { return a.v <= b; }
template <int K>
__host__ __device__ inline bool operator>=(const Dual<K> &a, double b) { return a.v >= b; }

// d sqrt(x) = dx / (2 sqrt(x)); the derivative is taken as 0 at x = 0, where
// it only multiplies vanishing gradients (the normal n = grad phi / |grad phi|).
template <int K>
__host__ __device__ inline Dual<K> sqrt(const Dual<K> &a) {
    Dual<K> r;
    r.v = ::sqrt(a.v);
    const double h = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.d[i] * h;
    return r;
}

template <int K>
__host__ __device__ inline double value(const Dual<K> &a) { return a.v; }
__host__ __device__ inline double value(double a) { return a; }
__host__ __device__ inline float value(float a) { return a; }

}  // namespace fcd
