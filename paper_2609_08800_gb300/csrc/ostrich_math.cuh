// Small-vector, quaternion and forward-mode dual-number helpers for the Ostrich kernels.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace ost {

// ---------------------------------------------------------------------------
// forward-mode dual number: value and one directional derivative
// ---------------------------------------------------------------------------
template <class T> struct dual {
  T v, d;
  __device__ __forceinline__ dual() {}
  __device__ __forceinline__ dual(T a) : v(a), d(T(0)) {}
  __device__ __forceinline__ dual(T a, T b) : v(a), d(b) {}
};
template <class T> __device__ __forceinline__ dual<T> operator+(dual<T> a, dual<T> b) { return dual<T>(a.v + b.v, a.d + b.d); }
template <class T> __device__ __forceinline__ dual<T> operator-(dual<T> a, dual<T> b) { return dual<T>(a.v - b.v, a.d - b.d); }
template <class T> __device__ __forceinline__ dual<T> operator-(dual<T> a) { return dual<T>(-a.v, -a.d); }
template <class T> __device__ __forceinline__ dual<T> operator*(dual<T> a, dual<T> b) { return dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> __device__ __forceinline__ dual<T> operator/(dual<T> a, dual<T> b) {
  T inv = T(1) / b.v;
  return dual<T>(a.v * inv, (a.d - a.v * inv * b.d) * inv);
}
template <class T> __device__ __forceinline__ dual<T> operator+(dual<T> a, T b) { return dual<T>(a.v + b, a.d); }
template <class T> __device__ __forceinline__ dual<T> operator+(T a, dual<T> b) { return dual<T>(a + b.v, b.d); }
template <class T> __device__ __forceinline__ dual<T> operator-(dual<T> a, T b) { return dual<T>(a.v - b, a.d); }
template <class T> __device__ __forceinline__ dual<T> operator-(T a, dual<T> b) { return dual<T>(a - b.v, -b.d); }
template <class T> __device__ __forceinline__ dual<T> operator*(dual<T> a, T b) { return dual<T>(a.v * b, a.d * b); }
template <class T> __device__ __forceinline__ dual<T> operator*(T a, dual<T> b) { return dual<T>(a * b.v, a * b.d); }
template <class T> __device__ __forceinline__ dual<T> operator/(dual<T> a, T b) { T inv = T(1) / b; return dual<T>(a.v * inv, a.d * inv); }

__device__ __forceinline__ float ssqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double ssqrt(double x) { return sqrt(x); }
template <class T> __device__ __forceinline__ dual<T> ssqrt(dual<T> a) {
  T s = ssqrt(a.v);
  return dual<T>(s, a.d / (T(2) * s));
}
// 1 / sqrt(x) of a Cholesky pivot: the hardware reciprocal square root in FP32 (within
// 2 ulp, one instruction instead of a rounded square root and a rounded division), the
// correctly rounded square root and quotient in FP64
__device__ __forceinline__ float pivot_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double pivot_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float sval(float x) { return x; }
__device__ __forceinline__ double sval(double x) { return x; }
template <class T> __device__ __forceinline__ T sval(dual<T> x) { return x.v; }

// ---------------------------------------------------------------------------
// 3-vectors
// ---------------------------------------------------------------------------
template <class S> struct vec3 { S x, y, z; };
template <class S> __device__ __forceinline__ vec3<S> v3(S a, S b, S c) { vec3<S> r; r.x = a; r.y = b; r.z = c; return r; }
template <class S> __device__ __forceinline__ vec3<S> operator+(vec3<S> a, vec3<S> b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class S> __device__ __forceinline__ vec3<S> operator-(vec3<S> a, vec3<S> b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class S, class K> __device__ __forceinline__ vec3<S> scale(vec3<S> a, K s) { return v3(a.x * s, a.y * s, a.z * s); }
template <class S> __device__ __forceinline__ S dot3(vec3<S> a, vec3<S> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> __device__ __forceinline__ vec3<S> cross3(vec3<S> a, vec3<S> b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class S, class T> __device__ __forceinline__ vec3<S> lift(vec3<T> a) { return v3(S(a.x), S(a.y), S(a.z)); }
// a . b with b of another scalar type (a dual vector against a constant one)
template <class S, class T> __device__ __forceinline__ S dotm(vec3<S> a, vec3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Rotate v by the normalised quaternion q/|q| = (w, x, y, z):  v + w t + qv x t, t = 2 qv x v.
template <class S> __device__ __forceinline__ vec3<S> qrot(const S* q, vec3<S> v) {
  S n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  S inv = S(1) / ssqrt(n2);
  S w = q[0] * inv;
  vec3<S> qv = v3(q[1] * inv, q[2] * inv, q[3] * inv);
  vec3<S> t = cross3(qv, v);
  t = v3(t.x + t.x, t.y + t.y, t.z + t.z);
  vec3<S> c = cross3(qv, t);
  return v3(v.x + w * t.x + c.x, v.y + w * t.y + c.y, v.z + w * t.z + c.z);
}

// Rotation matrix (row-major) of q/|q|, built by rotating the unit axes.
template <class S> __device__ __forceinline__ void qmat(const S* q, S* R) {
  vec3<S> ex = qrot(q, v3(S(1), S(0), S(0)));
  vec3<S> ey = qrot(q, v3(S(0), S(1), S(0)));
  vec3<S> ez = qrot(q, v3(S(0), S(0), S(1)));
  R[0] = ex.x; R[1] = ey.x; R[2] = ez.x;
  R[3] = ex.y; R[4] = ey.y; R[5] = ez.y;
  R[6] = ex.z; R[7] = ey.z; R[8] = ez.z;
}
template <class S, class M> __device__ __forceinline__ vec3<S> mat3(const M* R, vec3<S> v) {
  return v3(R[0] * v.x + R[1] * v.y + R[2] * v.z, R[3] * v.x + R[4] * v.y + R[5] * v.z,
            R[6] * v.x + R[7] * v.y + R[8] * v.z);
}
template <class S, class M> __device__ __forceinline__ vec3<S> mat3T(const M* R, vec3<S> v) {
  return v3(R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
            R[2] * v.x + R[5] * v.y + R[8] * v.z);
}

// Backward-Euler position update of one body, Eq. (1): p + h v, quat + h/2 (0, w) (x) quat.
template <class S, class U> __device__ __forceinline__ void kin_body(const S* qm, const U* u, double h, S* qp) {
  qp[0] = qm[0] + S(h) * u[0];
  qp[1] = qm[1] + S(h) * u[1];
  qp[2] = qm[2] + S(h) * u[2];
  S hh = S(0.5 * h);
  S wx = S(u[3]), wy = S(u[4]), wz = S(u[5]);
  S qw = qm[3], qx = qm[4], qy = qm[5], qz = qm[6];
  qp[3] = qw - hh * (wx * qx + wy * qy + wz * qz);
  qp[4] = qx + hh * (wx * qw + wy * qz - wz * qy);
  qp[5] = qy + hh * (wy * qw + wz * qx - wx * qz);
  qp[6] = qz + hh * (wz * qw + wx * qy - wy * qx);
}

// Angular part of a row Jacobian mapped through the rotation-rate map of Eq. (1):
// E^T a with E = (I + h/2 [wk]x) / (1 + (h/2)^2 |wk|^2).
// The same map with its scalar 1 / (1 + (h/2)^2 |wk|^2) formed once, for the rows of one
// body that share wk (the quotient is the costly part).
template <class T> struct MapE {
  vec3<T> wk;
  T hh, inv;
  __device__ __forceinline__ MapE(vec3<T> w, double h) : wk(w) {
    hh = T(0.5 * h);
    const T den = T(1) + hh * hh * (wk.x * wk.x + wk.y * wk.y + wk.z * wk.z);
    inv = T(1) / den;
  }
  template <class S> __device__ __forceinline__ vec3<S> operator()(vec3<S> a) const {
    const vec3<S> c = cross3(a, lift<S>(wk));
    return v3((a.x + c.x * hh) * inv, (a.y + c.y * hh) * inv, (a.z + c.z * hh) * inv);
  }
  // the transposed map: (E a) . v = a . (E^T v), with (a x w) . v = a . (w x v)
  __device__ __forceinline__ vec3<T> T_(vec3<T> v) const {
    const vec3<T> c = cross3(wk, v);
    return v3((v.x + c.x * hh) * inv, (v.y + c.y * hh) * inv, (v.z + c.z * hh) * inv);
  }
};
template <class S, class T> __device__ __forceinline__ vec3<S> map_Et(vec3<S> a, vec3<T> wk, double h) {
  return MapE<T>(wk, h)(a);
}

// ---------------------------------------------------------------------------
// compensated accumulation: sum of exact products (TwoProduct by fma) and exact
// partial sums (TwoSum), so a sum whose terms cancel keeps its accuracy.  The
// explicitly rounded intrinsics keep the compiler from fusing the pieces.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class T> struct acc2 {
  T s, c;
  __device__ __forceinline__ acc2() : s(T(0)), c(T(0)) {}
  __device__ __forceinline__ void add(T p) {
    T t = rn_add(s, p);
    T bp = rn_sub(t, s);
    T e = rn_add(rn_sub(s, rn_sub(t, bp)), rn_sub(p, bp));
    s = t;
    c = rn_add(c, e);
  }
  __device__ __forceinline__ void add_prod(T x, T y) {
    T p = rn_mul(x, y);
    T ep = rn_fma(x, y, -p);
    add(p);
    c = rn_add(c, ep);
  }
  __device__ __forceinline__ T value() const { return rn_add(s, c); }
};

}  // namespace ost
