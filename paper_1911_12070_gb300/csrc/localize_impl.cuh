// localize_impl.cuh -- device code of plaquette localization (Sec. 3.3.3,
// Eq. 6): the zero of the bilinear interpolant of a pierced face, shared by
// the stand-alone localization kernel, the batch localization kernel and the
// learned locator's plain fallback.  Products that feed an addition are
// rounded explicitly (__fmul_rn / __fadd_rn or fmaf), so the compiler cannot
// contract them differently in different kernels: every entry point gives
// the same samples bit for bit.
//
// Eq. 6 asks for x* = argmin rho(x), rho = |Phi|^2 (Eq. 3), with Phi linearly
// interpolated between nodes (Sec. 5).  Restricted to a pierced plaquette with
// corners P0..P3 in loop order at face coordinates (0,0) (1,0) (1,1) (0,1), the
// interpolant is F(u,v) = a + b u + c v + d u v with a = P0, b = P1 - P0,
// c = P3 - P0, d = P2 - P1 - P3 + P0.  When W = +-1 it has exactly one zero in
// the face (the two bilinear curves Re F = 0 and Im F = 0 meet at most twice,
// and the local degrees inside sum to W), so the minimiser is that zero and
// the minimum is 0.  It is found in FP32: eliminating u (then v) from
// F = 0 leaves a quadratic in v (u), every root gives a candidate, each
// candidate is refined by three Newton steps on (Re F, Im F), and the in-face
// candidate with the smallest |F| wins.
#pragma once

#include "qtv_internal.cuh"

namespace qtv {
namespace loc {

struct C2 {
  float x, y;
};
__device__ __forceinline__ C2 mk(float x, float y) { return C2{x, y}; }
__device__ __forceinline__ C2 sub(C2 p, C2 q) { return mk(p.x - q.x, p.y - q.y); }
// Im(p conj q)
__device__ __forceinline__ float crs(C2 p, C2 q) { return fmaf(p.y, q.x, __fmul_rn(-p.x, q.y)); }
// Re(p conj q)
__device__ __forceinline__ float dtr(C2 p, C2 q) { return fmaf(p.x, q.x, __fmul_rn(p.y, q.y)); }

// real roots of q2 t^2 + q1 t + q0 (0, 1 or 2 of them)
__device__ __forceinline__ int roots2(float q2, float q1, float q0, float& t0, float& t1) {
  const float scale = fabsf(q2) + fabsf(q1) + fabsf(q0);
  if (!(scale > 0.f)) return 0;
  if (fabsf(q2) <= 1e-6f * scale) {
    if (q1 == 0.f) return 0;
    t0 = -q0 / q1;
    return 1;
  }
  float disc = fmaf(q1, q1, __fmul_rn(__fmul_rn(-4.f, q2), q0));
  if (disc < 0.f) {
    if (disc > -1e-5f * q1 * q1) disc = 0.f;
    else return 0;
  }
  const float sq = sqrtf(disc);
  const float qq = -0.5f * (q1 + copysignf(sq, q1));
  if (qq == 0.f) {
    t0 = 0.f;
    return 1;
  }
  t0 = qq / q2;
  t1 = q0 / qq;
  return 2;
}

struct Bil {
  C2 a, b, c, d;
};

__device__ __forceinline__ C2 eval(const Bil& F, float u, float v) {
  // a + u (b + v d) + v c
  const C2 bv = mk(fmaf(v, F.d.x, F.b.x), fmaf(v, F.d.y, F.b.y));
  return mk(fmaf(u, bv.x, fmaf(v, F.c.x, F.a.x)), fmaf(u, bv.y, fmaf(v, F.c.y, F.a.y)));
}

__device__ __forceinline__ void newton(const Bil& F, float& u, float& v) {
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const C2 f = eval(F, u, v);
    const C2 fu = mk(fmaf(v, F.d.x, F.b.x), fmaf(v, F.d.y, F.b.y));
    const C2 fv = mk(fmaf(u, F.d.x, F.c.x), fmaf(u, F.d.y, F.c.y));
    const float det = fmaf(fu.x, fv.y, __fmul_rn(-fv.x, fu.y));
    if (det == 0.f) return;
    const float inv = 1.f / det;
    // explicit roundings: the same result in every kernel this is inlined
    // into (no context-dependent multiply-add contraction)
    const float du = __fmul_rn(-fmaf(fv.y, f.x, __fmul_rn(-fv.x, f.y)), inv);
    const float dv = __fmul_rn(-fmaf(fu.x, f.y, __fmul_rn(-fu.y, f.x)), inv);
    u = __fadd_rn(u, du);
    v = __fadd_rn(v, dv);
  }
}

// returns true if a zero was found inside the face
__device__ __forceinline__ bool solve_face(const C2 P[4], float& uo, float& vo, float& f2o) {
  Bil F;
  F.a = P[0];
  F.b = sub(P[1], P[0]);
  F.c = sub(P[3], P[0]);
  F.d = sub(sub(P[2], P[1]), F.c);
  float bu = 0.5f, bv = 0.5f, best = 3.4e38f;
  bool found = false;
  auto consider = [&](float u, float v) {
    if (!(u >= -0.05f && u <= 1.05f && v >= -0.05f && v <= 1.05f)) return;
    newton(F, u, v);
    if (!(u >= -1e-4f && u <= 1.f + 1e-4f && v >= -1e-4f && v <= 1.f + 1e-4f)) return;
    const C2 f = eval(F, u, v);
    const float f2 = fmaf(f.x, f.x, __fmul_rn(f.y, f.y));
    if (f2 < best) {
      best = f2;
      bu = u;
      bv = v;
      found = true;
    }
  };
  float t0 = 0.f, t1 = 0.f;
  // eliminate u: (a + c v) + u (b + d v) = 0, u real <=> Im(p conj q) = 0
  int nr = roots2(crs(F.c, F.d), __fadd_rn(crs(F.a, F.d), crs(F.c, F.b)), crs(F.a, F.b), t0, t1);
  for (int r = 0; r < nr; ++r) {
    const float v = r ? t1 : t0;
    const C2 p = mk(fmaf(v, F.c.x, F.a.x), fmaf(v, F.c.y, F.a.y));
    const C2 q = mk(fmaf(v, F.d.x, F.b.x), fmaf(v, F.d.y, F.b.y));
    const float qq = dtr(q, q);
    if (qq > 0.f) consider(-dtr(p, q) / qq, v);
  }
  if (!found) {
    // eliminate v: (a + b u) + v (c + d u) = 0
    nr = roots2(crs(F.b, F.d), __fadd_rn(crs(F.a, F.d), crs(F.b, F.c)), crs(F.a, F.c), t0, t1);
    for (int r = 0; r < nr; ++r) {
      const float u = r ? t1 : t0;
      const C2 p = mk(fmaf(u, F.b.x, F.a.x), fmaf(u, F.b.y, F.a.y));
      const C2 q = mk(fmaf(u, F.d.x, F.c.x), fmaf(u, F.d.y, F.c.y));
      const float qq = dtr(q, q);
      if (qq > 0.f) consider(u, -dtr(p, q) / qq);
    }
  }
  if (!found) {
    const C2 f = eval(F, 0.5f, 0.5f);
    best = fmaf(f.x, f.x, __fmul_rn(f.y, f.y));
  }
  uo = bu;
  vo = bv;
  f2o = best;
  return found;
}


// A face's grid position and corner values (the loads of its localization).
struct FaceIn {
  long long i, j, k;
  int o;
  bool exists;
  C2 P[4];
};

__device__ __forceinline__ void face_load(const float2* __restrict__ psi, int nx, int ny, int nz,
                                          unsigned long long id, FaceIn& F) {
  const int o = (int)(id & 3u);
  const unsigned long long lin = id >> 2;
  split_lin(lin, nx, ny, F.i, F.j, F.k);
  F.o = o;
  const long long sx = 1, sy = nx, sz = (long long)nx * ny;
  long long du, dv;  // strides of the face axes u, v
  bool exists;
  if (o == 0) { du = sx; dv = sy; exists = F.i + 1 < nx && F.j + 1 < ny; }
  else if (o == 1) { du = sy; dv = sz; exists = F.j + 1 < ny && F.k + 1 < nz; }
  else { du = sz; dv = sx; exists = F.k + 1 < nz && F.i + 1 < nx; }
  F.exists = o != 3 && exists && F.k < nz;
  if (!F.exists) return;  // not a face of this grid: touch no node
  const long long base = (long long)lin;
  const float2 p0 = __ldg(psi + base), p1 = __ldg(psi + base + du);
  const float2 p2 = __ldg(psi + base + du + dv), p3 = __ldg(psi + base + dv);
  F.P[0] = mk(p0.x, p0.y);
  F.P[1] = mk(p1.x, p1.y);
  F.P[2] = mk(p2.x, p2.y);
  F.P[3] = mk(p3.x, p3.y);
}

// The zero of a loaded face: position (grid coordinates scaled by h and
// shifted by the origin), residual, flags.
__device__ __forceinline__ void face_solve(const FaceIn& F, int wv, float h, float ox, float oy,
                                           float oz, float* xyz, float* resid, uint8_t* flags) {
  if (!F.exists) {
    xyz[0] = xyz[1] = xyz[2] = __int_as_float(0x7fc00000);
    *resid = __int_as_float(0x7fc00000);
    *flags = QTV_FLAG_ANOMALOUS;
    return;
  }
  float u, v, f2;
  const bool ok = solve_face(F.P, u, v, f2);
  uint8_t fl = 0;
  if (!ok || (wv != 1 && wv != -1)) fl |= QTV_FLAG_ANOMALOUS;
  float gx = (float)F.i, gy = (float)F.j, gz = (float)F.k;
  if (F.o == 0) { gx = __fadd_rn(gx, u); gy = __fadd_rn(gy, v); }
  else if (F.o == 1) { gy = __fadd_rn(gy, u); gz = __fadd_rn(gz, v); }
  else { gz = __fadd_rn(gz, u); gx = __fadd_rn(gx, v); }
  xyz[0] = fmaf(h, gx, ox);
  xyz[1] = fmaf(h, gy, oy);
  xyz[2] = fmaf(h, gz, oz);
  *resid = f2;
  *flags = fl;
}

// Localize one face given its id, winding and the field.
__device__ __forceinline__ void localize_face(const float2* __restrict__ psi, int nx, int ny, int nz,
                                              float h, float ox, float oy, float oz,
                                              unsigned long long id, int wv, float* xyz,
                                              float* resid, uint8_t* flags) {
  FaceIn F;
  face_load(psi, nx, ny, nz, id, F);
  face_solve(F, wv, h, ox, oy, oz, xyz, resid, flags);
}

}  // namespace loc
}  // namespace qtv
