// Per-cell arithmetic shared by the sweep kernels: 16-byte vector loads and stores of the four
// Legendre moments, and the closed-form solve of the frame-local 4x4 upwind DG-Q1 system
// (sigma_t I + a_x K (x) I + a_y I (x) K) psi = rhs, K = [[1, sqrt3], [-sqrt3, 3]], by block
// elimination over the y-modes with K^2 = 4 K - 6 I:  M = x I + y K and
// M^{-1} = ((x + 4y) I - y K) / (x^2 + 4xy + 6y^2)  (Sec. 2.2, App. B operators).
#pragma once

namespace rte {

__device__ __forceinline__ void load4(const float* p, float& a, float& b, float& c, float& d) {
    float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load4(const double* p, double& a, double& b, double& c, double& d) {
    double2 v0 = reinterpret_cast<const double2*>(p)[0];
    double2 v1 = reinterpret_cast<const double2*>(p)[1];
    a = v0.x; b = v0.y; c = v1.x; d = v1.y;
}
__device__ __forceinline__ void store4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double* p, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// Reciprocal of the 4x4 determinant (IEEE round-to-nearest in both precisions; on this part
// the correctly rounded FP32 reciprocal measured faster inside the sweep than the bare
// hardware approximation issued through inline PTX).
template <typename T>
__device__ __forceinline__ T rcp_exact(T v) { return T(1) / v; }
template <>
__device__ __forceinline__ float rcp_exact<float>(float v) { return __frcp_rn(v); }

// Closed-form solve of the frame-local 4x4 system (see the file header).
template <typename T>
__device__ __forceinline__ void cell_solve(T sig, T ax, T ay, T s3, T f0, T f1, T g0, T g1,
                                           T& u0, T& u1, T& v0, T& v1) {
    const T alpha = sig + ay;
    const T gamma = sig + T(3) * ay;
    const T beta = s3 * ay;
    const T x = fma(alpha, gamma, T(3) * ay * ay - T(6) * ax * ax);
    const T y = (alpha + gamma + T(4) * ax) * ax;
    const T c1 = fma(T(4), y, x);
    const T rdet = rcp_exact(fma(x, c1, T(6) * y * y));
    // w1 = gamma f + ax K f - beta g ;  w2 = alpha g + ax K g + beta f
    const T kf0 = fma(s3, f1, f0), kf1 = fma(T(3), f1, -s3 * f0);
    const T kg0 = fma(s3, g1, g0), kg1 = fma(T(3), g1, -s3 * g0);
    const T w10 = fma(gamma, f0, fma(ax, kf0, -beta * g0));
    const T w11 = fma(gamma, f1, fma(ax, kf1, -beta * g1));
    const T w20 = fma(alpha, g0, fma(ax, kg0, beta * f0));
    const T w21 = fma(alpha, g1, fma(ax, kg1, beta * f1));
    // M^{-1} w = ((x + 4y) w - y K w) / det
    const T kw10 = fma(s3, w11, w10), kw11 = fma(T(3), w11, -s3 * w10);
    const T kw20 = fma(s3, w21, w20), kw21 = fma(T(3), w21, -s3 * w20);
    u0 = fma(c1, w10, -y * kw10) * rdet;
    u1 = fma(c1, w11, -y * kw11) * rdet;
    v0 = fma(c1, w20, -y * kw20) * rdet;
    v1 = fma(c1, w21, -y * kw21) * rdet;
}

}  // namespace rte
