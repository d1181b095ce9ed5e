// cm_math.cuh -- FP32 device arithmetic of the smooth contact manifold (arXiv 2602.20304).
//
// Everything a CUDA thread computes for one vertex or one edge pair: the smooth
// operators of Sec. III, the SDF primitives of Sec. IV-B, the regularised E-E
// box QP with its smoothed analytic active set (Sec. IV-D2) and the signed
// witness quantities (Sec. IV-D3).  Transcendentals go to the MUFU pipe
// through ex2.approx / lg2.approx / rcp.approx / rsqrt.approx.
#pragma once

#include <cstdint>
#include <cmath>

#if defined(__CUDACC__)
#define CM_HD __host__ __device__ __forceinline__
// Functions of rarely taken paths (kept inline: an out-of-line call inside the hot
// loops cost more in register allocation than it saved in code size).
#define CM_HD_OUTLINE static __host__ __device__ __forceinline__
#else
#define CM_HD inline
#define CM_HD_OUTLINE static inline
#endif

namespace cm {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// ---------------------------------------------------------------- MUFU wrappers
CM_HD float ex2(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return exp2f(x);
#endif
}
CM_HD float lg2(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return log2f(x);
#endif
}
CM_HD float rcp(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / x;
#endif
}
CM_HD float rsq(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / sqrtf(x);
#endif
}
CM_HD float sqrt_(float x) {
#if defined(__CUDA_ARCH__)
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return sqrtf(x);
#endif
}
CM_HD float exp_(float x) { return ex2(x * kLog2e); }

// ---------------------------------------------------------------- 3-vectors
struct V3 {
  float x, y, z;
};
CM_HD V3 v3(float x, float y, float z) { return V3{x, y, z}; }
CM_HD V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
CM_HD V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
CM_HD V3 operator-(V3 a) { return v3(-a.x, -a.y, -a.z); }
CM_HD V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
CM_HD V3 operator*(V3 a, float s) { return v3(s * a.x, s * a.y, s * a.z); }
CM_HD V3& operator+=(V3& a, V3 b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  return a;
}
CM_HD float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
CM_HD V3 cross(V3 a, V3 b) {
  return v3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
CM_HD V3 fma3(float s, V3 a, V3 b) { return v3(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)); }

// Row-major 3x3 rotation.
struct M3 {
  float m[9];
};
CM_HD V3 mul(const M3& R, V3 v) {
  return v3(fmaf(R.m[0], v.x, fmaf(R.m[1], v.y, R.m[2] * v.z)),
            fmaf(R.m[3], v.x, fmaf(R.m[4], v.y, R.m[5] * v.z)),
            fmaf(R.m[6], v.x, fmaf(R.m[7], v.y, R.m[8] * v.z)));
}
CM_HD V3 mulT(const M3& R, V3 v) {
  return v3(fmaf(R.m[0], v.x, fmaf(R.m[3], v.y, R.m[6] * v.z)),
            fmaf(R.m[1], v.x, fmaf(R.m[4], v.y, R.m[7] * v.z)),
            fmaf(R.m[2], v.x, fmaf(R.m[5], v.y, R.m[8] * v.z)));
}
// Rotation of the normalised quaternion (w, x, y, z).
CM_HD M3 quat_rot(float w, float x, float y, float z) {
  float s = 1.0f / sqrtf(w * w + x * x + y * y + z * z);
  w *= s; x *= s; y *= s; z *= s;
  M3 R;
  R.m[0] = 1.f - 2.f * (y * y + z * z); R.m[1] = 2.f * (x * y - w * z); R.m[2] = 2.f * (x * z + w * y);
  R.m[3] = 2.f * (x * y + w * z); R.m[4] = 1.f - 2.f * (x * x + z * z); R.m[5] = 2.f * (y * z - w * x);
  R.m[6] = 2.f * (x * z - w * y); R.m[7] = 2.f * (y * z + w * x); R.m[8] = 1.f - 2.f * (x * x + y * y);
  return R;
}
// A^T B
CM_HD M3 mulTM(const M3& A, const M3& B) {
  M3 C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C.m[i * 3 + j] = A.m[0 * 3 + i] * B.m[0 * 3 + j] + A.m[1 * 3 + i] * B.m[1 * 3 + j] +
                       A.m[2 * 3 + i] * B.m[2 * 3 + j];
  return C;
}

// ---------------------------------------------------------------- smooth operators (Sec. III)
CM_HD float sigmoid(float x) { return rcp(1.0f + exp_(-x)); }
// log(1 + e^x) as max(x, 0) + log(1 + e^-|x|)
CM_HD float softplus(float x) { return fmaxf(x, 0.0f) + kLn2 * lg2(1.0f + exp_(-fabsf(x))); }
// eps softplus(x / eps) = max(x, 0) + eps ln(1 + e^-|x|/eps), in base 2
CM_HD float relu_s(float x, float inv_eps, float eps) {
  return fmaxf(x, 0.0f) + (eps * kLn2) * lg2(1.0f + ex2(-fabsf(x) * (inv_eps * kLog2e)));
}
CM_HD float clip_s(float x, float lo, float hi, float inv_eps, float eps) {
  return lo + relu_s(x - lo, inv_eps, eps) - relu_s(x - hi, inv_eps, eps);
}
// tanh(x) = 1 - 2 / (e^{2x} + 1); saturates cleanly to +-1.
CM_HD float tanh_(float x) { return 1.0f - 2.0f * rcp(exp_(2.0f * x) + 1.0f); }
// tanh(x / tau) given k2 = log2(e) / tau
CM_HD float tanh_k(float x, float k2) { return 1.0f - 2.0f * rcp(ex2(x * (2.0f * k2)) + 1.0f); }
// sigmoid(x / tau) given k2 = log2(e) / tau
CM_HD float sigmoid_k(float x, float k2) { return rcp(1.0f + ex2(-x * k2)); }
CM_HD float within01(float x, float inv_eps) { return sigmoid(x * inv_eps) * sigmoid((1.0f - x) * inv_eps); }

struct Params {
  float tau, w_reg, eps_clip, eps_min, eps_comp;
  int K, flags;
  int top_verts, top_edges;  // soft pre-selection counts (0: all)
  int trace_iters;           // sphere-tracing steps of E-E witnesses (0: off)
};

// ---------------------------------------------------------------- geometry kinds
enum Kind : int { kBox = 0, kCapsule = 1, kCylinder = 2, kEllipsoid = 3, kHull = 4, kSqUnion = 5 };

// Local vertex of a template row u = (u_x, u_y, u_z, s) for the given dims.
CM_HD V3 map_vertex(int kind, float ux, float uy, float uz, float s, V3 d) {
  switch (kind) {
    case kBox:
    case kEllipsoid: return v3(d.x * ux, d.y * uy, d.z * uz);
    case kCylinder: return v3(d.x * ux, d.x * uy, d.y * uz);
    case kCapsule: return v3(d.x * ux, d.x * uy, fmaf(d.x, uz, s * d.y));
    default: return v3(ux, uy, uz);
  }
}

// SDF value and the gradient its normal is built from (grad phi; grad f for the
// superquadric), in the body's local frame.
struct Sdf {
  float phi;
  V3 g;
};

// Box: convex polyhedron of the planes +-y_i - h_i (Sec. IV-B2).
CM_HD Sdf sdf_box(V3 y, V3 h, float tau, float inv_tau) {
  float px = y.x - h.x, nx = -y.x - h.x, py = y.y - h.y, ny = -y.y - h.y, pz = y.z - h.z,
        nz = -y.z - h.z;
  float m = fmaxf(fmaxf(fmaxf(px, nx), fmaxf(py, ny)), fmaxf(pz, nz));
  float k = inv_tau * kLog2e;
  float epx = ex2((px - m) * k), enx = ex2((nx - m) * k), epy = ex2((py - m) * k),
        eny = ex2((ny - m) * k), epz = ex2((pz - m) * k), enz = ex2((nz - m) * k);
  float S = ((epx + enx) + (epy + eny)) + (epz + enz);
  float r = rcp(S);
  Sdf o;
  o.phi = m + tau * kLn2 * lg2(S);
  o.g = v3((epx - enx) * r, (epy - eny) * r, (epz - enz) * r);
  return o;
}

// ---------------------------------------------------------------- packed FP32x2
CM_HD float2 ffma2(float2 a, float2 b, float2 c) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
  return __ffma2_rn(a, b, c);
#else
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
CM_HD float2 fadd2(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
CM_HD float2 dup2(float a) { return make_float2(a, a); }

// Convex polyhedron given by planes (n, o): phi = LSE_tau of n . y - o (Sec. IV-B2).
// The planes arrive pre-scaled by k = log2(e) / tau, (k n, k o), so a plane value
// is already the exponent in base 2; phi = tau ln2 (m + log2 S) and the gradient
// sum_f pi_f n_f is rescaled by 1/k = tau ln2.  Single pass over the planes in
// chunks of 4 with an online maximum (a rescale only when the maximum grows).
CM_HD Sdf sdf_planes(V3 y, const float4* P, int nP, float tau, float /*inv_tau*/) {
  float m = -3.0e38f, S = 0.f;
  V3 G = v3(0.f, 0.f, 0.f);
  for (int f0 = 0; f0 < nP; f0 += 4) {
    float z[4];
    float4 q[4];
    float cm = m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + j;
      q[j] = f < nP ? P[f] : make_float4(0.f, 0.f, 0.f, 3.0e38f);
      z[j] = fmaf(q[j].x, y.x, fmaf(q[j].y, y.y, fmaf(q[j].z, y.z, -q[j].w)));
      cm = fmaxf(cm, z[j]);
    }
    if (cm > m) {
      const float r = ex2(m - cm);
      S *= r;
      G = G * r;
      m = cm;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float e = ex2(z[j] - m);
      S += e;
      G.x = fmaf(e, q[j].x, G.x);
      G.y = fmaf(e, q[j].y, G.y);
      G.z = fmaf(e, q[j].z, G.z);
    }
  }
  const float t = tau * kLn2;
  Sdf o;
  o.phi = t * (m + lg2(S));
  o.g = G * (t * rcp(S));
  return o;
}

// The same LSE at two points at once: the value at y1 and the gradient at y2
// (the two uses an edge pair makes of one body's SDF).  Each plane is loaded
// once and both plane values come from packed FP32x2 FMAs.
CM_HD void sdf_planes2(V3 y1, V3 y2, const float4* P, int nP, float tau, Sdf& o1, Sdf& o2) {
  const float2 X = make_float2(y1.x, y2.x), Y = make_float2(y1.y, y2.y), Z = make_float2(y1.z, y2.z);
  float2 m = dup2(-3.0e38f), S = dup2(0.f);
  V3 G = v3(0.f, 0.f, 0.f);
  for (int f0 = 0; f0 < nP; f0 += 4) {
    float2 z[4];
    float4 q[4];
    float2 cm = m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + j;
      q[j] = f < nP ? P[f] : make_float4(0.f, 0.f, 0.f, 3.0e38f);
      z[j] = ffma2(dup2(q[j].x), X, ffma2(dup2(q[j].y), Y, ffma2(dup2(q[j].z), Z, dup2(-q[j].w))));
      cm.x = fmaxf(cm.x, z[j].x);
      cm.y = fmaxf(cm.y, z[j].y);
    }
    if (cm.x > m.x || cm.y > m.y) {
      const float r1 = ex2(m.x - cm.x), r2 = ex2(m.y - cm.y);
      S = make_float2(S.x * r1, S.y * r2);
      G = G * r2;
      m = cm;
    }
    const float2 nm = make_float2(-m.x, -m.y);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 d = fadd2(z[j], nm);
      const float2 e = make_float2(ex2(d.x), ex2(d.y));
      S = fadd2(S, e);
      G.x = fmaf(e.y, q[j].x, G.x);
      G.y = fmaf(e.y, q[j].y, G.y);
      G.z = fmaf(e.y, q[j].z, G.z);
    }
  }
  const float t = tau * kLn2;
  o1.phi = t * (m.x + lg2(S.x));
  o1.g = v3(0.f, 0.f, 0.f);
  o2.phi = t * (m.y + lg2(S.y));
  o2.g = G * (t * rcp(S.y));
}

// The same LSE at two points with what its reverse needs, so that the adjoint
// makes one pass over the planes instead of two: value and gradient at y1, and
// value, gradient and Hessian at y2.  With pi_f = softmax_f(s_f / tau) the
// gradient is g = sum_f pi_f n_f and the Hessian H = (sum_f pi_f n_f n_f^T - g g^T) / tau,
// so the plane-by-plane reverse sum_f pi_f (phibar + gbar . (n_f - g) / tau) n_f
// equals phibar g + H gbar.  In the pre-scaled planes (k n, k o), k = log2(e) / tau,
// with S = sum e_f, G = sum e_f (k n_f), Mq = sum e_f (k n_f)(k n_f)^T:
// g = (tau ln2) G / S and H = tau ln2^2 (Mq / S - (G / S)(G / S)^T).  H is returned
// as (xx, xy, xz, yy, yz, zz).  Chunks of 4 planes with an online maximum per point.
CM_HD void sdf_planes2_h(V3 y1, V3 y2, const float4* P, int nP, float tau, Sdf& o1, Sdf& o2, float (&H)[6]) {
  const float2 X = make_float2(y1.x, y2.x), Y = make_float2(y1.y, y2.y), Z = make_float2(y1.z, y2.z);
  float2 m = dup2(-3.0e38f), S = dup2(0.f);
  float2 Gx = dup2(0.f), Gy = dup2(0.f), Gz = dup2(0.f);  // (point 1, point 2)
  float2 Mxx_yy = dup2(0.f), Mxy_yz = dup2(0.f), Mxz_zz = dup2(0.f);
  for (int f0 = 0; f0 < nP; f0 += 4) {
    float2 z[4];
    float4 q[4];
    float2 cm = m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + j;
      q[j] = f < nP ? P[f] : make_float4(0.f, 0.f, 0.f, 3.0e38f);
      z[j] = ffma2(dup2(q[j].x), X, ffma2(dup2(q[j].y), Y, ffma2(dup2(q[j].z), Z, dup2(-q[j].w))));
      cm.x = fmaxf(cm.x, z[j].x);
      cm.y = fmaxf(cm.y, z[j].y);
    }
    if (cm.x > m.x || cm.y > m.y) {
      const float2 r = make_float2(ex2(m.x - cm.x), ex2(m.y - cm.y));
      S = make_float2(S.x * r.x, S.y * r.y);
      Gx = make_float2(Gx.x * r.x, Gx.y * r.y);
      Gy = make_float2(Gy.x * r.x, Gy.y * r.y);
      Gz = make_float2(Gz.x * r.x, Gz.y * r.y);
      Mxx_yy = make_float2(Mxx_yy.x * r.y, Mxx_yy.y * r.y);
      Mxy_yz = make_float2(Mxy_yz.x * r.y, Mxy_yz.y * r.y);
      Mxz_zz = make_float2(Mxz_zz.x * r.y, Mxz_zz.y * r.y);
      m = cm;
    }
    const float2 nm = make_float2(-m.x, -m.y);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 d = fadd2(z[j], nm);
      const float2 e = make_float2(ex2(d.x), ex2(d.y));
      S = fadd2(S, e);
      Gx = ffma2(e, dup2(q[j].x), Gx);
      Gy = ffma2(e, dup2(q[j].y), Gy);
      Gz = ffma2(e, dup2(q[j].z), Gz);
      const float2 txy = make_float2(e.y * q[j].x, e.y * q[j].y);
      const float tz = e.y * q[j].z;
      Mxx_yy = ffma2(txy, make_float2(q[j].x, q[j].y), Mxx_yy);
      Mxy_yz = ffma2(txy, make_float2(q[j].y, q[j].z), Mxy_yz);
      Mxz_zz = ffma2(make_float2(txy.x, tz), make_float2(q[j].z, q[j].z), Mxz_zz);
    }
  }
  const float t = tau * kLn2;
  const float i1 = rcp(S.x), i2 = rcp(S.y);
  o1.phi = t * (m.x + lg2(S.x));
  o1.g = v3(Gx.x, Gy.x, Gz.x) * (t * i1);
  o2.phi = t * (m.y + lg2(S.y));
  const V3 gh = v3(Gx.y * i2, Gy.y * i2, Gz.y * i2);  // G / S at y2, scaled units
  o2.g = gh * t;
  const float h = t * kLn2;
  H[0] = h * fmaf(Mxx_yy.x, i2, -gh.x * gh.x);
  H[1] = h * fmaf(Mxy_yz.x, i2, -gh.x * gh.y);
  H[2] = h * fmaf(Mxz_zz.x, i2, -gh.x * gh.z);
  H[3] = h * fmaf(Mxx_yy.y, i2, -gh.y * gh.y);
  H[4] = h * fmaf(Mxy_yz.y, i2, -gh.y * gh.z);
  H[5] = h * fmaf(Mxz_zz.y, i2, -gh.z * gh.z);
}

// sdf_planes2_h without a shift, for an edge pair whose y2 is the body's own witness
// within a scaled distance of 60 of its own edge (the condition of sdf_planes_ee):
// the sums at y2 then stay within 2^-60 .. nP 2^60, and every plane term is added
// as it is read, with no running maximum.  At y1 (the other body's witness) the
// plain sum S1 may overflow to +inf or underflow to 0; phi(y1) = tau ln S1 is then
// +inf or -inf, so sigma(-phi(y1)/tau) is exactly 0 or 1 with derivative 0, and
// the gradient at y1, which only multiplies that derivative, is returned as 0
// whenever S1 lies outside 2^-100 .. 2^100 (there sigma' < 2^-100 / tau).
CM_HD void sdf_planes2_h_ee(V3 y1, V3 y2, const float4* P, int nP, float tau, Sdf& o1, Sdf& o2,
                            float (&H)[6]) {
  const float2 X = make_float2(y1.x, y2.x), Y = make_float2(y1.y, y2.y), Z = make_float2(y1.z, y2.z);
  float2 S = dup2(0.f), Gx = dup2(0.f), Gy = dup2(0.f), Gz = dup2(0.f);
  float2 Mxx_yy = dup2(0.f), Mxy_yz = dup2(0.f), Mxz_zz = dup2(0.f);
#pragma unroll 4
  for (int f = 0; f < nP; ++f) {
    const float4 q = P[f];
    const float2 z = ffma2(dup2(q.x), X, ffma2(dup2(q.y), Y, ffma2(dup2(q.z), Z, dup2(-q.w))));
    const float2 e = make_float2(ex2(z.x), ex2(z.y));
    S = fadd2(S, e);
    Gx = ffma2(e, dup2(q.x), Gx);
    Gy = ffma2(e, dup2(q.y), Gy);
    Gz = ffma2(e, dup2(q.z), Gz);
    const float2 txy = make_float2(e.y * q.x, e.y * q.y);
    const float tz = e.y * q.z;
    Mxx_yy = ffma2(txy, make_float2(q.x, q.y), Mxx_yy);
    Mxy_yz = ffma2(txy, make_float2(q.y, q.z), Mxy_yz);
    Mxz_zz = ffma2(make_float2(txy.x, tz), make_float2(q.z, q.z), Mxz_zz);
  }
  const float t = tau * kLn2;
  o1.phi = t * lg2(S.x);
  const bool in1 = S.x >= 0x1p-100f && S.x <= 0x1p100f;
  o1.g = in1 ? v3(Gx.x, Gy.x, Gz.x) * (t * rcp(S.x)) : v3(0.f, 0.f, 0.f);
  const float i2 = rcp(S.y);
  o2.phi = t * lg2(S.y);
  const V3 gh = v3(Gx.y * i2, Gy.y * i2, Gz.y * i2);  // G / S at y2, scaled units
  o2.g = gh * t;
  const float h = t * kLn2;
  H[0] = h * fmaf(Mxx_yy.x, i2, -gh.x * gh.x);
  H[1] = h * fmaf(Mxy_yz.x, i2, -gh.x * gh.y);
  H[2] = h * fmaf(Mxz_zz.x, i2, -gh.x * gh.z);
  H[3] = h * fmaf(Mxx_yy.y, i2, -gh.y * gh.y);
  H[4] = h * fmaf(Mxy_yz.y, i2, -gh.y * gh.z);
  H[5] = h * fmaf(Mxz_zz.y, i2, -gh.z * gh.z);
}

// One point of sdf_planes2_h: value, gradient and Hessian (xx, xy, xz, yy, yz, zz).
CM_HD void sdf_planes_h(V3 y, const float4* P, int nP, float tau, Sdf& o, float (&H)[6]) {
  float m = -3.0e38f, S = 0.f;
  V3 G = v3(0.f, 0.f, 0.f);
  float M[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int f0 = 0; f0 < nP; f0 += 4) {
    float z[4];
    float4 q[4];
    float cm = m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + j;
      q[j] = f < nP ? P[f] : make_float4(0.f, 0.f, 0.f, 3.0e38f);
      z[j] = fmaf(q[j].x, y.x, fmaf(q[j].y, y.y, fmaf(q[j].z, y.z, -q[j].w)));
      cm = fmaxf(cm, z[j]);
    }
    if (cm > m) {
      const float r = ex2(m - cm);
      S *= r;
      G = G * r;
#pragma unroll
      for (int c = 0; c < 6; ++c) M[c] *= r;
      m = cm;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float e = ex2(z[j] - m);
      S += e;
      const V3 t = v3(e * q[j].x, e * q[j].y, e * q[j].z);
      G += t;
      M[0] = fmaf(t.x, q[j].x, M[0]);
      M[1] = fmaf(t.x, q[j].y, M[1]);
      M[2] = fmaf(t.x, q[j].z, M[2]);
      M[3] = fmaf(t.y, q[j].y, M[3]);
      M[4] = fmaf(t.y, q[j].z, M[4]);
      M[5] = fmaf(t.z, q[j].z, M[5]);
    }
  }
  const float t = tau * kLn2, iS = rcp(S), h = t * kLn2;
  const V3 gh = G * iS;
  o.phi = t * (m + lg2(S));
  o.g = gh * t;
  H[0] = h * fmaf(M[0], iS, -gh.x * gh.x);
  H[1] = h * fmaf(M[1], iS, -gh.x * gh.y);
  H[2] = h * fmaf(M[2], iS, -gh.x * gh.z);
  H[3] = h * fmaf(M[3], iS, -gh.y * gh.y);
  H[4] = h * fmaf(M[4], iS, -gh.y * gh.z);
  H[5] = h * fmaf(M[5], iS, -gh.z * gh.z);
}

// What an edge pair's candidates take from a polyhedron's SDF (Sec. IV-D3):
// sigma(-phi(y1)/tau) at the other body's witness y1 and the gradient at the
// body's own witness y2 (for its normal), plus sigma(-phi(y2)/tau) for the
// pre-selection safeguard.  With the planes pre-scaled to base-2 exponents z_f,
// sigma(-phi/tau) = 1 / (1 + sum_f 2^z_f) exactly, so the plain (unshifted) sum
// serves: where it over- or underflows in FP32, sigma saturates to 0 or 1 the
// same way.  The gradient is the ratio G / S, whatever the shift.  The caller
// uses this only while y2 lies within a scaled distance of 60 of its own edge
// segment: every plane passes no closer than that bound above the segment and
// the planes through the edge lie no farther below, so S2 stays within
// 2^-60 .. nP 2^60.  Returns S1 = sum at y1, S2 = sum at y2 and G2 = grad phi(y2).
CM_HD void sdf_planes_ee(V3 y1, V3 y2, const float4* P, int nP, float tau, float& S1, float& S2,
                         V3& G2) {
  const float2 X = make_float2(y1.x, y2.x), Y = make_float2(y1.y, y2.y), Z = make_float2(y1.z, y2.z);
  float2 S = dup2(0.f);
  V3 G = v3(0.f, 0.f, 0.f);
#pragma unroll 4
  for (int f = 0; f < nP; ++f) {
    const float4 q = P[f];
    const float2 z = ffma2(dup2(q.x), X, ffma2(dup2(q.y), Y, ffma2(dup2(q.z), Z, dup2(-q.w))));
    const float2 e = make_float2(ex2(z.x), ex2(z.y));
    S = fadd2(S, e);
    G.x = fmaf(e.y, q.x, G.x);
    G.y = fmaf(e.y, q.y, G.y);
    G.z = fmaf(e.y, q.z, G.z);
  }
  S1 = S.x;
  S2 = S.y;
  G2 = G * (tau * kLn2 * rcp(S.y));
}

// Superquadric with eps1 = eps2 = 1 (Sec. IV-B1): phi = |y| (1 - f^-1/2), f = |y~|^2;
// the normal comes from grad f = 2 y / d^2.
CM_HD Sdf sdf_ellipsoid(V3 y, V3 d) {
  V3 id = v3(rcp(d.x), rcp(d.y), rcp(d.z));
  V3 yt = v3(y.x * id.x, y.y * id.y, y.z * id.z);
  float f = dot(yt, yt);
  float r = sqrt_(dot(y, y));
  Sdf o;
  o.phi = r - r * rsq(f);
  o.g = v3(2.f * yt.x * id.x, 2.f * yt.y * id.y, 2.f * yt.z * id.z);
  return o;
}

// Capsule of radius r around the z segment [-h, h] with a soft-clipped axial
// coordinate: phi = |y - clip_s(y_z, -h, h) z| - r.
// The soft clip's two softplus terms and their sigmoids share e^-|x| per side:
// softplus(x) = max(x, 0) + ln(1 + e^-|x|), sigmoid(x) = (x >= 0 ? 1 : e^-|x|) / (1 + e^-|x|),
// and the difference of the two logarithms is the logarithm of a ratio.
CM_HD Sdf sdf_capsule(V3 y, float rad, float h, float tau, float inv_tau) {
  float up = (y.z + h) * inv_tau, dn = (y.z - h) * inv_tau;
  const float Eu = exp_(-fabsf(up)), Ed = exp_(-fabsf(dn));
  const float iu = rcp(1.f + Eu), id = rcp(1.f + Ed);
  float c = -h + tau * ((fmaxf(up, 0.f) - fmaxf(dn, 0.f)) + kLn2 * lg2((1.f + Eu) * id));
  V3 w = v3(y.x, y.y, y.z - c);
  float r2 = dot(w, w);
  float ir = r2 > 0.f ? rsq(r2) : 0.f;
  float r = r2 * ir;
  float dc = (up >= 0.f ? iu : Eu * iu) - (dn >= 0.f ? id : Ed * id);
  Sdf o;
  o.phi = r - rad;
  o.g = v3(w.x * ir, w.y * ir, w.z * (1.f - dc) * ir);
  return o;
}

// Cylinder of radius r and half-height h along z: LSE_tau(rho - r, z - h, -z - h).
CM_HD Sdf sdf_cylinder(V3 y, float rad, float h, float tau, float inv_tau) {
  float rho2 = y.x * y.x + y.y * y.y;
  float irho = rho2 > 0.f ? rsq(rho2) : 0.f;
  float rho = rho2 * irho;
  float s0 = rho - rad, s1 = y.z - h, s2 = -y.z - h;
  float m = fmaxf(s0, fmaxf(s1, s2));
  float k = inv_tau * kLog2e;
  float e0 = ex2((s0 - m) * k), e1 = ex2((s1 - m) * k), e2 = ex2((s2 - m) * k);
  float S = e0 + e1 + e2;
  float ri = rcp(S);
  Sdf o;
  o.phi = m + tau * kLn2 * lg2(S);
  float a = e0 * ri * irho;
  o.g = v3(a * y.x, a * y.y, (e1 - e2) * ri);
  return o;
}

// log2(2^a + 2^b) without forming either power.
CM_HD float log2_add(float a, float b) { return fmaxf(a, b) + lg2(1.f + ex2(-fabsf(a - b))); }

// Smooth union of superquadrics (Sec. IV-B, IV-B1).  Five rows per primitive:
// (M row 0, c_0), (M row 1, c_1), (M row 2, c_2) with x = M y + c its own-frame
// point (M = R^T, c = -R^T t), (1/a, 1/b, 1/c, p1 = 2/eps1) and (p2 = 2/eps2,
// r = eps2/eps1, h = eps1/2, -).  Per primitive, with x~ = x / (a, b, c):
//   s = |x~_x|^p2 + |x~_y|^p2, f = s^r + |x~_z|^p1, phi_l = (1 - f^-h) |x|,
//   d f / d x~_x = r p2 s^(r-1) |x~_x|^(p2-1) sgn x~_x  (likewise y),
//   d f / d x~_z = p1 |x~_z|^(p1-1) sgn x~_z.
// Everything is carried as base-2 logarithms (sums of powers by log2_add), so
// the large powers of a boxy primitive (2/eps up to 20) neither overflow nor
// underflow on the way; magnitudes are clamped away from 0 so that a point on
// a primitive's axis or centre stays finite.  The union
// phi = -tau ln sum_l exp(-phi_l / tau) is accumulated in one pass with a
// running minimum m; its normal gradient sum_l pi_l R_l grad_x f_l
// (pi = softmax(-phi / tau)) takes each weight into the exponent of the
// gradient components, so a negligible weight times a huge gradient is 0.
CM_HD Sdf sdf_sq_union(V3 y, const float4* P, int L, float tau, float inv_tau) {
  const float k = inv_tau * kLog2e;
  float m = 3.0e38f, S = 0.f;
  V3 G = v3(0.f, 0.f, 0.f);
  for (int l = 0; l < L; ++l) {
    const float4 r0 = P[5 * l], r1 = P[5 * l + 1], r2 = P[5 * l + 2], r3 = P[5 * l + 3], r4 = P[5 * l + 4];
    const V3 x = v3(fmaf(r0.x, y.x, fmaf(r0.y, y.y, fmaf(r0.z, y.z, r0.w))),
                    fmaf(r1.x, y.x, fmaf(r1.y, y.y, fmaf(r1.z, y.z, r1.w))),
                    fmaf(r2.x, y.x, fmaf(r2.y, y.y, fmaf(r2.z, y.z, r2.w))));
    const float xx = x.x * r3.x, xy = x.y * r3.y, xz = x.z * r3.z;
    const float p1 = r3.w, p2 = r4.x, rr = r4.y, h = r4.z;
    const float lx = lg2(fmaxf(fabsf(xx), 1e-20f)), ly = lg2(fmaxf(fabsf(xy), 1e-20f)),
                lz = lg2(fmaxf(fabsf(xz), 1e-20f));
    const float ls = log2_add(p2 * lx, p2 * ly);          // log2 s
    const float lf = log2_add(rr * ls, p1 * lz);          // log2 f
    const float phi = (1.f - ex2(-h * lf)) * sqrt_(dot(x, x));
    if (phi < m) {  // new running minimum: rescale what was summed relative to the old one
      const float sc = ex2((phi - m) * k);
      S *= sc;
      G = G * sc;
      m = phi;
    }
    const float le = (m - phi) * k;                        // log2 of the union weight
    S += ex2(le);
    const float ex = le + (rr - 1.f) * ls;
    const float gx = copysignf(rr * p2 * r3.x * ex2(ex + (p2 - 1.f) * lx), xx);
    const float gy = copysignf(rr * p2 * r3.y * ex2(ex + (p2 - 1.f) * ly), xy);
    const float gz = copysignf(p1 * r3.z * ex2(le + (p1 - 1.f) * lz), xz);
    G.x += fmaf(gx, r0.x, fmaf(gy, r1.x, gz * r2.x));
    G.y += fmaf(gx, r0.y, fmaf(gy, r1.y, gz * r2.y));
    G.z += fmaf(gx, r0.z, fmaf(gy, r1.z, gz * r2.z));
  }
  Sdf o;
  o.phi = m - tau * kLn2 * lg2(S);
  o.g = G * rcp(S);
  return o;
}

// Regularised normal g / sqrt(tau + |g|^2) (Sec. IV-B).
CM_HD V3 normal_of(V3 g, float tau) { return g * rsq(tau + dot(g, g)); }

// A body as seen by the kernels: its kind, the dims in use and its planes
// (hull planes pre-scaled by log2(e) / tau, see sdf_planes).
struct Body {
  int kind;
  V3 dims;
  const float4* planes;
  int n_planes;
};

CM_HD Sdf body_sdf(const Body& b, V3 y, float tau, float inv_tau) {
  switch (b.kind) {
    case kBox: return sdf_box(y, b.dims, tau, inv_tau);
    case kEllipsoid: return sdf_ellipsoid(y, b.dims);
    case kCapsule: return sdf_capsule(y, b.dims.x, b.dims.y, tau, inv_tau);
    case kCylinder: return sdf_cylinder(y, b.dims.x, b.dims.y, tau, inv_tau);
    case kSqUnion: return sdf_sq_union(y, b.planes, b.n_planes / 5, tau, inv_tau);
    default: return sdf_planes(y, b.planes, b.n_planes, tau, inv_tau);
  }
}

// A box, capsule, cylinder or ellipsoid: body_sdf without the polyhedron and
// superquadric branches (for code compiled for a known pair class).
CM_HD Sdf prim_sdf(const Body& b, V3 y, float tau, float inv_tau) {
  switch (b.kind) {
    case kBox: return sdf_box(y, b.dims, tau, inv_tau);
    case kEllipsoid: return sdf_ellipsoid(y, b.dims);
    case kCapsule: return sdf_capsule(y, b.dims.x, b.dims.y, tau, inv_tau);
    default: return sdf_cylinder(y, b.dims.x, b.dims.y, tau, inv_tau);
  }
}
// A body's SDF at two points: o1 for its value at y1, o2 for its gradient at y2.
CM_HD void body_sdf2(const Body& b, V3 y1, V3 y2, float tau, float inv_tau, Sdf& o1, Sdf& o2) {
  if (b.kind == kHull) {
    sdf_planes2(y1, y2, b.planes, b.n_planes, tau, o1, o2);
  } else {
    o1 = body_sdf(b, y1, tau, inv_tau);
    o2 = body_sdf(b, y2, tau, inv_tau);
  }
}

// Sphere tracing of a witness onto its own body's SDF surface (Supplement,
// mesh-SDF discrepancies): `iters` steps x <- x - phi(x) u along the fixed
// direction u = grad phi(x_0) / |grad phi(x_0)|, in the body's own frame.
CM_HD V3 trace_to_surface(const Body& b, V3 x, int iters, float tau, float it) {
  Sdf s = body_sdf(b, x, tau, it);
  const V3 u = s.g * rsq(dot(s.g, s.g));
  for (int i = 0; i < iters; ++i) {
    if (i) s = body_sdf(b, x, tau, it);
    x = fma3(-s.phi, u, x);
  }
  return x;
}

// ---------------------------------------------------------------- E-E witness QP (Sec. IV-D2)
// Box QP  min 1/2 a^T Q a + c^T a  on [0,1]^2 with Q = A^T A + lam I,
// c = A^T b - lam/2 (1, 1), A = [t1, t2], t1 = a1 - a0, t2 = b0 - b1, b = a0 - b0.
// The unconstrained minimiser uses the Lagrange / Binet-Cauchy forms
//   det Q  = |t1 x t2|^2 + lam (|t1|^2 + |t2|^2) + lam^2,
//   Q12 c2 - Q22 c1 = -(t1 x t2).(b x t2) + lam ((|t2|^2 - t1.t2)/2 - t1.b + lam/2),
//   Q12 c1 - Q11 c2 = -(t1 x t2).(t1 x b) + lam ((|t1|^2 - t1.t2)/2 - t2.b + lam/2),
// which equal the textbook 2x2 inverse but keep the FP32 cancellation of the
// near-parallel case inside one cross product.
struct QPOut {
  float a1, a2, con;
};

CM_HD float qp_cost(float Q11, float Q12, float Q22, float c1, float c2, float a1, float a2) {
  return 0.5f * (Q11 * a1 * a1 + 2.f * Q12 * a1 * a2 + Q22 * a2 * a2) + c1 * a1 + c2 * a2;
}

struct QPPre {  // quantities of the QP set-up, reused by the adjoint
  V3 t1, t2, b;
  float Q11, Q12, Q22, c1, c2;
};

CM_HD QPPre qp_setup(V3 a0, V3 a1, V3 b0, V3 b1, float lam) {
  QPPre q;
  q.t1 = a1 - a0;
  q.t2 = b0 - b1;
  q.b = a0 - b0;
  float T11 = dot(q.t1, q.t1), T12 = dot(q.t1, q.t2), T22 = dot(q.t2, q.t2);
  q.Q11 = T11 + lam;
  q.Q12 = T12;
  q.Q22 = T22 + lam;
  q.c1 = dot(q.t1, q.b) - 0.5f * lam;
  q.c2 = dot(q.t2, q.b) - 0.5f * lam;
  return q;
}

CM_HD QPOut qp_solve(const QPPre& q, float lam, const Params& p) {
  V3 X = cross(q.t1, q.t2);
  float T11 = q.Q11 - lam, T22 = q.Q22 - lam, T12 = q.Q12;
  float B1 = q.c1 + 0.5f * lam, B2 = q.c2 + 0.5f * lam;
  float det = dot(X, X) + lam * (T11 + T22) + lam * lam;
  float n1 = -dot(X, cross(q.b, q.t2)) + lam * (0.5f * (T22 - T12) - B1 + 0.5f * lam);
  float n2 = -dot(X, cross(q.t1, q.b)) + lam * (0.5f * (T11 - T12) - B2 + 0.5f * lam);
  float idet = rcp(det);
  float au1 = n1 * idet, au2 = n2 * idet;
  // minimisers along the four sides of the unit box, soft-clipped to [0, 1]
  float ie = rcp(p.eps_clip);
  float iQ11 = rcp(q.Q11), iQ22 = rcp(q.Q22);
  float s1 = clip_s(-(q.Q12 + q.c2) * iQ22, 0.f, 1.f, ie, p.eps_clip);  // a1 = 1
  float s2 = clip_s(-q.c2 * iQ22, 0.f, 1.f, ie, p.eps_clip);             // a1 = 0
  float s3 = clip_s(-(q.Q12 + q.c1) * iQ11, 0.f, 1.f, ie, p.eps_clip);  // a2 = 1
  float s4 = clip_s(-q.c1 * iQ11, 0.f, 1.f, ie, p.eps_clip);             // a2 = 0
  float J1 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, 1.f, s1);
  float J2 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, 0.f, s2);
  float J3 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, s3, 1.f);
  float J4 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, s4, 0.f);
  // soft argmin of the four costs
  float Jm = fminf(fminf(J1, J2), fminf(J3, J4));
  float k = -rcp(p.eps_min) * kLog2e;
  float w1 = ex2((J1 - Jm) * k), w2 = ex2((J2 - Jm) * k), w3 = ex2((J3 - Jm) * k),
        w4 = ex2((J4 - Jm) * k);
  float iw = rcp((w1 + w2) + (w3 + w4));
  float ac1 = (w1 + w3 * s3 + w4 * s4) * iw;
  float ac2 = (w1 * s1 + w2 * s2 + w3) * iw;
  // con = within01(au1) within01(au2), the four sigmoids under one reciprocal:
  // 1 / prod (1 + e^-x_i); a factor that overflows makes con 0, as it should.
  float ic = rcp(p.eps_comp);
  float con = rcp(((1.f + exp_(-au1 * ic)) * (1.f + exp_((au1 - 1.f) * ic))) *
                  ((1.f + exp_(-au2 * ic)) * (1.f + exp_((au2 - 1.f) * ic))));
  QPOut o;
  o.a1 = fmaf(con, au1 - ac1, ac1);
  o.a2 = fmaf(con, au2 - ac2, ac2);
  o.con = con;
  return o;
}

// The same active set without smoothing (the paper's Ours-NS, Sec. V): the side
// minimisers clipped to [0, 1], the argmin of the four costs (first on ties) and
// con the inclusive test 0 <= au <= 1 of both coordinates.
CM_HD QPOut qp_solve_hard(const QPPre& q, float lam) {
  V3 X = cross(q.t1, q.t2);
  float T11 = q.Q11 - lam, T22 = q.Q22 - lam, T12 = q.Q12;
  float B1 = q.c1 + 0.5f * lam, B2 = q.c2 + 0.5f * lam;
  float det = dot(X, X) + lam * (T11 + T22) + lam * lam;
  float n1 = -dot(X, cross(q.b, q.t2)) + lam * (0.5f * (T22 - T12) - B1 + 0.5f * lam);
  float n2 = -dot(X, cross(q.t1, q.b)) + lam * (0.5f * (T11 - T12) - B2 + 0.5f * lam);
  float idet = rcp(det);
  float au1 = n1 * idet, au2 = n2 * idet;
  QPOut o;
  if (au1 >= 0.f && au1 <= 1.f && au2 >= 0.f && au2 <= 1.f) {
    o.a1 = au1;
    o.a2 = au2;
    o.con = 1.f;
    return o;
  }
  float iQ11 = rcp(q.Q11), iQ22 = rcp(q.Q22);
  float s1 = fminf(fmaxf(-(q.Q12 + q.c2) * iQ22, 0.f), 1.f);  // a1 = 1
  float s2 = fminf(fmaxf(-q.c2 * iQ22, 0.f), 1.f);             // a1 = 0
  float s3 = fminf(fmaxf(-(q.Q12 + q.c1) * iQ11, 0.f), 1.f);  // a2 = 1
  float s4 = fminf(fmaxf(-q.c1 * iQ11, 0.f), 1.f);             // a2 = 0
  float J = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, 1.f, s1);
  o.a1 = 1.f;
  o.a2 = s1;
  const float J2 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, 0.f, s2);
  if (J2 < J) { J = J2; o.a1 = 0.f; o.a2 = s2; }
  const float J3 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, s3, 1.f);
  if (J3 < J) { J = J3; o.a1 = s3; o.a2 = 1.f; }
  const float J4 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, s4, 0.f);
  if (J4 < J) { o.a1 = s4; o.a2 = 0.f; }
  o.con = 0.f;
  return o;
}

// ---------------------------------------------------------------- V-F witness (Sec. IV-D1)
// Smoothed closest point of triangle (t0, t1, t2) to v: plane projection if the
// soft barycentric test says inside, else the soft-argmin blend of the three
// edge projections (edge parameter soft-clipped to [0, 1]).  Returns the
// witness and the inside indicator.
CM_HD V3 vf_witness(V3 v, V3 t0, V3 t1, V3 t2, const Params& p, float& inside) {
  const float ie = rcp(p.eps_clip);
  V3 q[3];
  float c[3];
  const V3 A[3] = {t0, t1, t0}, B[3] = {t1, t2, t2};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const V3 e = B[j] - A[j];
    const float s = clip_s(dot(v - A[j], e) * rcp(dot(e, e)), 0.f, 1.f, ie, p.eps_clip);
    q[j] = fma3(s, e, A[j]);
    const V3 d = v - q[j];
    c[j] = sqrt_(dot(d, d));
  }
  const float cm = fminf(c[0], fminf(c[1], c[2]));
  const float k = -rcp(p.eps_min) * kLog2e;
  const float w0 = ex2((c[0] - cm) * k), w1 = ex2((c[1] - cm) * k), w2 = ex2((c[2] - cm) * k);
  const float iw = rcp(w0 + w1 + w2);
  const V3 pc = (q[0] * w0 + q[1] * w1 + q[2] * w2) * iw;
  const V3 d10 = t1 - t0, d20 = t2 - t0;
  const V3 nb = cross(d10, d20);
  const float ia = rsq(dot(nb, nb));
  const V3 n = nb * ia;
  const V3 rel = v - t0;
  const V3 pr = rel - n * dot(rel, n);
  const float b2 = dot(cross(d10, pr), n) * ia, b1 = dot(cross(pr, d20), n) * ia, b0 = 1.f - b1 - b2;
  const float ic = rcp(p.eps_comp);
  inside = within01(b0, ic) * within01(b1, ic) * within01(b2, ic);
  const V3 pu = t0 + pr;
  return pc + (pu - pc) * inside;
}

// The same routine without smoothing (Ours-NS): edge parameters clipped to [0, 1],
// the nearest of the three edge points (first on ties), and the plane projection
// where all three barycentric coordinates lie in [0, 1].
CM_HD V3 vf_witness_hard(V3 v, V3 t0, V3 t1, V3 t2, float& inside) {
  const V3 d10 = t1 - t0, d20 = t2 - t0;
  const V3 nb = cross(d10, d20);
  const float ia = rsq(dot(nb, nb));
  const V3 n = nb * ia;
  const V3 rel = v - t0;
  const V3 pr = rel - n * dot(rel, n);
  const float b2 = dot(cross(d10, pr), n) * ia, b1 = dot(cross(pr, d20), n) * ia, b0 = 1.f - b1 - b2;
  if (b0 >= 0.f && b0 <= 1.f && b1 >= 0.f && b1 <= 1.f && b2 >= 0.f && b2 <= 1.f) {
    inside = 1.f;
    return t0 + pr;
  }
  inside = 0.f;
  const V3 A[3] = {t0, t1, t0}, B[3] = {t1, t2, t2};
  V3 best = t0;
  float bc = 3.0e38f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const V3 e = B[j] - A[j];
    const float s = fminf(fmaxf(dot(v - A[j], e) * rcp(dot(e, e)), 0.f), 1.f);
    const V3 q = fma3(s, e, A[j]);
    const V3 d = v - q;
    const float c = dot(d, d);
    if (c < bc) {
      bc = c;
      best = q;
    }
  }
  return best;
}

}  // namespace cm
