// Forward-mode dual numbers for the adjoint: a value and its derivatives with
// respect to M seeded inputs.  Instantiating the piece / projection templates
// of lift_device.cuh with Dual<M> yields the Jacobian of a projection with
// respect to the projected point and the data-term parameters; branch
// decisions are taken on the values, exactly as on the float path.
#pragma once

#include <cuda_runtime.h>

#include "lift_device.cuh"

namespace lift {

template <int M>
struct Dual {
    float v;
    float d[M];
    __device__ __forceinline__ Dual() : v(0.0f) {
#pragma unroll
        for (int j = 0; j < M; ++j) d[j] = 0.0f;
    }
    __device__ __forceinline__ Dual(float x) : v(x) {  // a constant
#pragma unroll
        for (int j = 0; j < M; ++j) d[j] = 0.0f;
    }
    __device__ __forceinline__ static Dual seed(float x, int j) {
        Dual r(x);
        r.d[j] = 1.0f;
        return r;
    }
};

template <int M> __device__ __forceinline__ float val(const Dual<M> &a) { return a.v; }

template <int M>
__device__ __forceinline__ Dual<M> operator+(const Dual<M> &a, const Dual<M> &b)
{
    Dual<M> r(a.v + b.v);
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = a.d[j] + b.d[j];
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M> operator-(const Dual<M> &a, const Dual<M> &b)
{
    Dual<M> r(a.v - b.v);
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = a.d[j] - b.d[j];
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M> operator-(const Dual<M> &a)
{
    Dual<M> r(-a.v);
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = -a.d[j];
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M> operator*(const Dual<M> &a, const Dual<M> &b)
{
    Dual<M> r(a.v * b.v);
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = a.d[j] * b.v + a.v * b.d[j];
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M> operator/(const Dual<M> &a, const Dual<M> &b)
{
    Dual<M> r(a.v / b.v);
    const float ib = 1.0f / b.v;
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = (a.d[j] - r.v * b.d[j]) * ib;
    return r;
}
template <int M> __device__ __forceinline__ Dual<M> operator+(const Dual<M> &a, float b) { return a + Dual<M>(b); }
template <int M> __device__ __forceinline__ Dual<M> operator+(float a, const Dual<M> &b) { return Dual<M>(a) + b; }
template <int M> __device__ __forceinline__ Dual<M> operator-(const Dual<M> &a, float b) { return a - Dual<M>(b); }
template <int M> __device__ __forceinline__ Dual<M> operator-(float a, const Dual<M> &b) { return Dual<M>(a) - b; }
template <int M>
__device__ __forceinline__ Dual<M> operator*(const Dual<M> &a, float b)
{
    Dual<M> r(a.v * b);
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = a.d[j] * b;
    return r;
}
template <int M> __device__ __forceinline__ Dual<M> operator*(float a, const Dual<M> &b) { return b * a; }
template <int M> __device__ __forceinline__ Dual<M> operator/(const Dual<M> &a, float b) { return a * (1.0f / b); }
template <int M> __device__ __forceinline__ Dual<M> operator/(float a, const Dual<M> &b) { return Dual<M>(a) / b; }

template <int M>
__device__ __forceinline__ Dual<M> tmin(const Dual<M> &a, const Dual<M> &b) { return a.v <= b.v ? a : b; }
template <int M>
__device__ __forceinline__ Dual<M> tmax(const Dual<M> &a, const Dual<M> &b) { return a.v >= b.v ? a : b; }
template <int M>
__device__ __forceinline__ Dual<M> tsqrt(const Dual<M> &a)
{
    Dual<M> r(sqrtf(a.v));
    const float g = r.v > 0.0f ? 0.5f / r.v : 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) r.d[j] = a.d[j] * g;
    return r;
}

}  // namespace lift
