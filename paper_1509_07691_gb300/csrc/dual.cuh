// dual.cuh -- forward-mode dual numbers v + d*eps (eps^2 = 0) for the
// curvature Jacobian of the adjoint: one derivative direction per lane.
// Comparisons act on the value, so branch decisions are those of the plain
// evaluation and every lane of a warp takes the same path.
#pragma once

#include <cuda_runtime.h>

namespace fslk {

template <typename S>
struct Dual {
    S v, d;
    Dual() = default;
    __host__ __device__ constexpr Dual(double a) : v(S(a)), d(S(0)) {}
    __host__ __device__ constexpr Dual(S a, S b, int) : v(a), d(b) {}

    friend __device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d, 0); }
    friend __device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d, 0); }
    friend __device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d, 0); }
    friend __device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d, 0); }
    friend __device__ __forceinline__ Dual operator/(Dual a, Dual b) {
        const S q = a.v / b.v;
        return Dual(q, (a.d - q * b.d) / b.v, 0);
    }
    __device__ __forceinline__ Dual &operator+=(Dual b) { return *this = *this + b; }
    __device__ __forceinline__ Dual &operator-=(Dual b) { return *this = *this - b; }
    __device__ __forceinline__ Dual &operator*=(Dual b) { return *this = *this * b; }
    __device__ __forceinline__ Dual &operator/=(Dual b) { return *this = *this / b; }
    friend __device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
    friend __device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
    friend __device__ __forceinline__ bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
    friend __device__ __forceinline__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
    friend __device__ __forceinline__ bool operator==(Dual a, Dual b) { return a.v == b.v; }
    friend __device__ __forceinline__ bool operator!=(Dual a, Dual b) { return a.v != b.v; }
    friend __device__ __forceinline__ Dual sqrt(Dual a) {
        const S r = sqrt(a.v);
        return Dual(r, r > S(0) ? a.d / (S(2) * r) : S(0), 0);
    }
    friend __device__ __forceinline__ Dual fabs(Dual a) { return a.v < S(0) ? -a : a; }
};

// value of a plain or dual number
__device__ __forceinline__ float value_of(float a) { return a; }
__device__ __forceinline__ double value_of(double a) { return a; }
template <typename S>
__device__ __forceinline__ S value_of(Dual<S> a) { return a.v; }

// 1/sqrt(x) (rsqrtf for float, as the forward normals use)
__device__ __forceinline__ float rsqrt_of(float a) { return rsqrtf(a); }
__device__ __forceinline__ double rsqrt_of(double a) { return rsqrt(a); }
template <typename S>
__device__ __forceinline__ Dual<S> rsqrt_of(Dual<S> a) {
    const S r = rsqrt_of(a.v);
    return Dual<S>(r, S(-0.5) * a.d * r * r * r, 0);
}

// plain scalar type underneath
template <typename T>
struct scalar_of { using type = T; };
template <typename S>
struct scalar_of<Dual<S>> { using type = S; };

}  // namespace fslk
