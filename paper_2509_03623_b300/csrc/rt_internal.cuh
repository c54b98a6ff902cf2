// Internal declarations of the B300 line radiative-transfer library: the per-launch
// parameter block (passed by value as a __grid_constant__ kernel argument, so a launch
// needs no device allocation or copy), fast-math device helpers, the per-ray setup and the
// field lookup shared by the forward and adjoint kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rt.h"

namespace rtb {

// Tabulated LTE opacity factor Phi(t) = log2[ f_l(T) (1 - exp(-dE/kT)) ], t = log2(T/K),
// f_l = g_l exp(-E_l/kT)/Z(T). Cubic Hermite segments stored as Horner coefficients.
constexpr int kTabN = 232;  // nodes t = 0, 1/16, ..., 14.4375 (1 K .. 22 kK)
constexpr float kTabT0 = 0.0f;
constexpr float kTabInvH = 16.0f;
constexpr int kTabSeg = kTabN - 1;

struct Ray;

// A double-float number: the unevaluated sum hi + lo of two FP32 numbers, |lo| <= ulp(hi) / 2
// (about 44 significant bits). The disk's ray setup runs in this arithmetic on the FP32 pipes
// (the FP64 pipe of this part retires about two lanes per clock per SM).
struct F2 {
  float hi, lo;
};

struct MarchParams {
  // grid
  int nr, nz, r_log, hard_edge;
  float lr_scale, lr_off;   // u = lg2(r^2/r_in^2)*lr_scale (log grid) or r*lr_scale+lr_off
  float r_in2, inv_rin2;    // r_in^2 [au^2] and its reciprocal
  float zr_max, w_scale;    // w = (z/r) * w_scale
  float zr_max2;            // zr_max^2 (gas test without a square root)
  const float *T, *n, *vt, *hlo, *hhi;
  const float *vphi;        // optional rotation field [km/s]; nullptr: Keplerian
  // 3-D Cartesian grid (rt_render3d; box != 0): chord box in double (ray setup), node
  // placement in float, packed node records {T, n, vt, x_co} and {vx, vy, vz, 0}
  int box;
  // the dense comparison march: every sample of a ray is visited (no gas range) and every
  // channel block is marched (no channel window)
  int full_range, no_window;
  double bx0, bx1, by0, by1, bz0, bz1;
  int n3x, n3y, n3z;
  // per axis: a node near the centre of the box (index k and position c [au]) and the nodes
  // per au; positions are measured from that node so that the fine FP32 resolution of small
  // coordinates reaches the interpolation weights where the fields change fastest
  int g3kx, g3ky, g3kz;
  float g3cx, g3cy, g3cz, g3sx, g3sy, g3sz;
  float cos_if;                              // cos i (FP32)
  const float4 *node_a, *node_b;
  // 3-D spherical grid (rt_render_sph; sph != 0): radial index from r^2 as for the
  // axisymmetric grid (r_log, lr_scale, lr_off, r_in2, inv_rin2), colatitude index
  // (theta - th0) th_scale, azimuth index phi ph_scale with phi = atan2(y, x) in [0, 2 pi);
  // node records node_a / node_b {T, n, vt, x_co} and {v_r, v_theta, v_phi, 0} in
  // [nph][nth][nr] order; rays are clipped to the sphere of radius R_cyl (= r_out)
  int sph, snr, snth, snph;
  float th0, th1, th_scale, ph_scale, r_out2;
  float sin_if;             // sin i (FP32, for v_los = v_phi x sin i / r)
  float x_co, edge_k;       // edge_k = log2(e) / edge_w
  int vturb_mach;
  float c_th, c_mach;       // alpha^2 [km^2 s^-2] = c_th T + vt^2  |  T (c_th + c_mach vt^2)
  // geometry (double: per-ray setup only); reciprocals of the ray direction's components
  // (omega = (0, sin i, -cos i); 0 where the component is 0), of 2 sin^2 i and of n_samples
  double sin_i, cos_i, cos_pa, sin_pa, R_cyl, H_cyl, px, py;
  double inv_wy, inv_wz, inv_2a, inv_ns;
  // the same constants as double-float numbers for the FP32 ray setup of the disk (f2_setup:
  // a disk view whose pixel indices are below 2^22), with H_cyl, R_cyl, R_cyl^2, 4 sin^2 i and
  // vk sin i
  F2 f_px, f_py, f_cos_pa, f_sin_pa, f_cos_i, f_sin_i, f_H, f_R, f_R2, f_4a, f_inv_wz,
      f_inv_2a, f_inv_ns, f_vks;
  int f2_setup;
  float vk;                 // sqrt(G M) [km s^-1 au^1/2]
  float vsys;
  // view
  int nx, ny, nch, n_samples;
  int step_bits;            // significant bits of the per-sample step (k * step exact)
  float out_scale, I0;
  // line
  float kappa_k;            // dtau (log2 units) = kappa_k n_CO 2^Phi inv_alpha ds
  float theta_s;            // (E_u - E_l)/k * log2(e) [K]
  int v_uniform;            // channel velocities equally spaced: v_c = v0 + c dv
  float v0, dv;
  // neural-field modulation per (pixel, sample): {o0, o1, o2, o3} with T e^{o0}, n e^{o1},
  // h_lo + h_scale o2, h_hi + h_scale o3; nullptr for grid fields alone
  const float4 *mod;
  float h_scale;
  // optional work counters (device; nullptr for none). Forward kernel, 2 x u64: samples with
  // gas whose physics was evaluated, channel evaluations computed. Adjoint kernel, 4 x u64:
  // samples with gas, evaluations of the forward pass, 0 (a recompute pass of an earlier
  // design), evaluations of the reverse pass.
  unsigned long long *work;
  // optional corner quads (pack_cells): per grid cell (i, j) the four nodes its bilinear
  // interpolation reads, {f(i,j), f(i+1,j), f(i,j+1), f(i+1,j+1)}, for T, n_H2, v_turb and
  // the rotation field when there is one (three or four float4 per cell, cells in [j][i]
  // order), and per radial interval i
  // {h_lo(i), h_lo(i+1), h_hi(i), h_hi(i+1)}: four 16-byte loads per sample instead of 16
  // scalar ones. nullptr: the kernels read the node arrays (same values, same rounding).
  const float4 *cell, *hcell;
  // optional dynamic work distribution of the forward march (nullptr: each warp takes a fixed
  // interleaved share of the work units and sets up its rays itself): the ray setups of
  // every pixel from a pre-pass, and a launch-wide counter (zeroed before the launch) from
  // which warps take work units one at a time
  const Ray *rays;
  unsigned *unit_ctr;
  float v[RT_MAX_CH];
  float tab[kTabSeg * 4];
};

// ---------------------------------------------------------------------------------------
// Hardware approximations (MUFU). ex2 runs at 32/clk/SM on B300, the others at 16/clk/SM.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// square root to about 2^-23 relative (one MUFU operation instead of the correctly rounded
// sequence of sqrtf)
__device__ __forceinline__ float sqa(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-ray setup: pixel -> ray origin on the sky plane and chord through the cylinder, in
// double precision (once per ray). Sample positions are then formed in FP32 from a high
// part of the step with few enough significant bits that k * step is exact, so a position
// carries about one rounding of its own magnitude.
struct Ray {
  float x;                 // constant disk-frame x along the ray
  float yb, zb, yb2, zb2;  // first-sample position (midpoint of segment 0), high + low parts
  float dy, dz, dy2, dz2;  // step per sample, high part + remainder
  float ds;                // segment length [au]
  float vfac;              // sqrt(GM) sin i x  [km s^-1 au^{1/2}]
  int hit;                 // ray crosses the bounding cylinder
  int pix;                 // pixel index iy * nx + ix
  int klo, khi;            // samples that can hold gas: klo..khi (khi < klo: none)
};

// Round v to `bits` significant bits (scalings by powers of two are exact, so no division).
__host__ __device__ __forceinline__ double round_bits(double v, int bits) {
  if (v == 0.0) return 0.0;
  int e;
  frexp(v, &e);
  return ldexp(nearbyint(ldexp(v, bits - e)), e - bits);
}

__device__ __forceinline__ float sample_coord(float kf, float base, float base2, float step,
                                              float step2) {
  return fmaf(kf, step, base) + fmaf(kf, step2, base2);
}

// Samples of a ray that can lie inside the gas wedge |z| <= zr_max r: the hull of
// {s in [lo, hi] : zr_max^2 (x^2 + y(s)^2) - z(s)^2 >= 0} (a quadratic in s), widened by two
// segments plus 2e-3 of the ray's coordinate magnitude (far above the FP32 rounding of the
// roots, which is largest for rays grazing the wedge) and turned into sample indices. Every
// sample outside the range fails the per-sample gas test, so marching only the range gives
// the same cube. FP32 arithmetic, once per ray.
__device__ __forceinline__ void gas_range(const MarchParams &P, float xs, float y0, float z0,
                                          float wy, float wz, float lo, float hi, int *klo,
                                          int *khi) {
  const float m2 = P.zr_max2;
  const float A = m2 * wy * wy - wz * wz;
  const float B = 2.0f * (m2 * y0 * wy - z0 * wz);
  const float C = m2 * fmaf(xs, xs, y0 * y0) - z0 * z0;
  float s1 = lo, s2 = hi;
  if (A == 0.0f) {  // linear: B s + C >= 0 (B = 0 as well: the whole chord)
    if (B > 0.0f) s1 = fmaxf(lo, -C / B);
    else if (B < 0.0f) s2 = fminf(hi, -C / B);
  } else {
    const float disc = B * B - 4.0f * A * C;
    if (disc <= 0.0f) {
      // A > 0: gas along the whole chord; A < 0: at most near the tangent point (the pad
      // below covers a discriminant that rounded to zero or below)
      if (A < 0.0f) s1 = s2 = -B / (2.0f * A);
    } else {
      const float q = -0.5f * (B + copysignf(sqrtf(disc), B));
      float r1 = q / A, r2 = q != 0.0f ? C / q : r1;
      if (r1 > r2) {
        const float t = r1;
        r1 = r2;
        r2 = t;
      }
      if (A < 0.0f) {  // gas between the roots
        s1 = fmaxf(lo, r1);
        s2 = fminf(hi, r2);
      } else {  // gas outside (r1, r2): hull of the two pieces inside the chord
        s1 = lo <= r1 ? lo : fmaxf(lo, r2);
        s2 = hi >= r2 ? hi : fminf(hi, r1);
      }
    }
  }
  const int n = P.n_samples;
  const float ds = (hi - lo) / (float)n;
  const float pad = 2.0f * ds + 2e-3f * (fabsf(lo) + fabsf(hi) + fabsf(xs) + fabsf(y0) + fabsf(z0));
  s1 = fmaxf(s1 - pad, lo);
  s2 = fminf(s2 + pad, hi);
  // (fmaxf / fminf take lo / hi for a NaN bound: the whole ray)
  if (!(s1 <= s2 && ds > 0.0f)) {  // the widened hull misses the chord: no gas
    *klo = 0;
    *khi = -1;
    return;
  }
  // sample k sits at s = lo + (k + 1/2) ds
  const float f1 = fmaxf((s1 - lo) / ds - 0.5f, 0.0f), f2 = fminf((s2 - lo) / ds - 0.5f, (float)n);
  *klo = (int)floorf(f1);
  *khi = min((int)ceilf(f2), n - 1);
}

// Double-float arithmetic: error-free transformations of a sum (Knuth's TwoSum; Dekker's
// Fast2Sum, for |a| >= |b|) and of a product (one FMA), and the double-word sum, product and
// square root built from them (Dekker 1971; Joldes, Muller and Popescu 2017: relative errors
// of a few 2^-48 for the sum and product).
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  return F2{s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  const F2 v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2{-a.hi, -a.lo}; }
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) { return f2_add(a, f2_neg(b)); }
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);  // a.hi b.hi - p exactly
  return fast_two_sum(p, __fadd_rn(e, __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.lo))));
}
__device__ __forceinline__ F2 f2_mul1(F2 a, float b) {  // by an FP32 number
  const float p = __fmul_rn(a.hi, b);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
__device__ __forceinline__ F2 f2_scale(F2 a, float pow2) {  // by a power of two (exact)
  return F2{a.hi * pow2, a.lo * pow2};
}
// square root of a >= 0: the FP32 root of the high part plus one correction from the exact
// residual a - s^2 (s^2 by the product transformation; a.hi - s^2 rounded is exact)
__device__ __forceinline__ F2 f2_sqrt(F2 a) {
  if (!(a.hi > 0.0f)) return F2{0.0f, 0.0f};
  const float s = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s, s), e = __fmaf_rn(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  return fast_two_sum(s, __fmul_rn(r, 0.5f * rcp(s)));
}
__device__ __forceinline__ bool f2_lt(F2 a, F2 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// Round v to `bits` significant bits (FP32).
__device__ __forceinline__ float round_bits_f(float v, int bits) {
  if (v == 0.0f) return 0.0f;
  int e;
  frexpf(v, &e);
  return ldexpf(rintf(ldexpf(v, bits - e)), e - bits);
}

// The disk's ray setup (setup_ray below) in double-float arithmetic: the same steps and the
// same Ray, with the start point and step carried to about 2^-44 relative instead of FP64's
// 2^-53 (the FP32 sample positions built from them round once to their own magnitude either
// way).
__device__ __forceinline__ Ray setup_ray_f2(const MarchParams &P, int ix, int iy, bool active) {
  Ray R;
  // pixel centre offsets (i + 1/2 - n/2), exact in FP32 below 2^22 pixels a side
  const float cx = ((float)ix + 0.5f) - 0.5f * (float)P.nx;
  const float cy = ((float)iy + 0.5f) - 0.5f * (float)P.ny;
  const F2 X = f2_mul1(P.f_px, cx), Y = f2_mul1(P.f_py, cy);
  const F2 xs = f2_add(f2_mul(X, P.f_cos_pa), f2_mul(Y, P.f_sin_pa));
  const F2 ys = f2_sub(f2_mul(Y, P.f_cos_pa), f2_mul(X, P.f_sin_pa));
  const F2 P0y = f2_mul(ys, P.f_cos_i), P0z = f2_mul(ys, P.f_sin_i);
  const F2 wy = P.f_sin_i, wz = f2_neg(P.f_cos_i);
  F2 lo = F2{-INFINITY, 0.0f}, hi = F2{INFINITY, 0.0f};
  bool ok = active;
  if (wz.hi != 0.0f) {  // the slab |z| <= H_cyl
    const F2 t1 = f2_mul(f2_sub(f2_neg(P.f_H), P0z), P.f_inv_wz);
    const F2 t2 = f2_mul(f2_sub(P.f_H, P0z), P.f_inv_wz);
    const bool o = f2_lt(t1, t2);
    lo = o ? t1 : t2;
    hi = o ? t2 : t1;
  } else if (f2_lt(P.f_H, F2{fabsf(P0z.hi), P0z.hi < 0.0f ? -P0z.lo : P0z.lo})) {
    ok = false;
  }
  const F2 c = f2_sub(f2_add(f2_mul(xs, xs), f2_mul(P0y, P0y)), P.f_R2);
  if (wy.hi != 0.0f) {
    // the cylinder r <= R_cyl: roots of a s^2 + b s + c, a = wy^2, b = 2 P0y wy, with the
    // discriminant 4 a (R - x)(R + x)
    const F2 b = f2_scale(f2_mul(P0y, wy), 2.0f);
    const F2 disc = f2_mul(P.f_4a, f2_mul(f2_sub(P.f_R, xs), f2_add(P.f_R, xs)));
    if (disc.hi < 0.0f) {
      ok = false;
    } else {
      const F2 sq = f2_sqrt(disc);
      const F2 r1 = f2_mul(f2_sub(f2_neg(b), sq), P.f_inv_2a);
      const F2 r2 = f2_mul(f2_sub(sq, b), P.f_inv_2a);
      if (f2_lt(lo, r1)) lo = r1;
      if (f2_lt(r2, hi)) hi = r2;
    }
  } else if (c.hi > 0.0f || (c.hi == 0.0f && c.lo > 0.0f)) {
    ok = false;
  }
  ok = ok && f2_lt(lo, hi);
  if (!ok) {
    lo = F2{0.0f, 0.0f};
    hi = F2{0.0f, 0.0f};
  }
  const F2 ds = f2_mul(f2_sub(hi, lo), P.f_inv_ns);
  const F2 s0 = f2_add(lo, f2_scale(ds, 0.5f));
  const F2 yb = f2_add(P0y, f2_mul(s0, wy)), zb = f2_add(P0z, f2_mul(s0, wz));
  const F2 dy = f2_mul(ds, wy), dz = f2_mul(ds, wz);
  R.x = xs.hi;
  R.yb = yb.hi;
  R.yb2 = yb.lo;
  R.zb = zb.hi;
  R.zb2 = zb.lo;
  const float dyh = round_bits_f(dy.hi, P.step_bits), dzh = round_bits_f(dz.hi, P.step_bits);
  R.dy = dyh;
  R.dy2 = __fadd_rn(__fsub_rn(dy.hi, dyh), dy.lo);
  R.dz = dzh;
  R.dz2 = __fadd_rn(__fsub_rn(dz.hi, dzh), dz.lo);
  R.ds = ds.hi;
  R.vfac = f2_mul(P.f_vks, xs).hi;
  R.hit = ok ? 1 : 0;
  R.pix = iy * P.nx + ix;
  R.klo = 0;
  R.khi = ok ? P.n_samples - 1 : -1;
  if (ok && !P.full_range)
    gas_range(P, xs.hi, P0y.hi, P0z.hi, wy.hi, wz.hi, lo.hi, hi.hi, &R.klo, &R.khi);
  return R;
}

__device__ __forceinline__ Ray setup_ray(const MarchParams &P, int ix, int iy, bool active) {
  if (P.f2_setup) return setup_ray_f2(P, ix, iy, active);
  Ray R;
  double X = ((double)ix + 0.5 - 0.5 * P.nx) * P.px;
  double Y = ((double)iy + 0.5 - 0.5 * P.ny) * P.py;
  double xs = X * P.cos_pa + Y * P.sin_pa;
  double ys = -X * P.sin_pa + Y * P.cos_pa;
  double P0y = ys * P.cos_i, P0z = ys * P.sin_i;
  double wy = P.sin_i, wz = -P.cos_i;
  double lo = -1e300, hi = 1e300;
  bool ok = active;
  if (P.sph) {
    // chord through the sphere r <= R_cyl: |P0 + s omega|^2 = R_cyl^2 with |omega| = 1
    const double b = P0y * wy + P0z * wz;
    const double c = xs * xs + P0y * P0y + P0z * P0z - P.R_cyl * P.R_cyl;
    const double disc = b * b - c;
    if (!(disc > 0.0)) {
      ok = false;
    } else {
      const double sq = sqrt(disc);
      lo = -b - sq;
      hi = -b + sq;
    }
  } else if (P.box) {
    // chord through the box, slab by slab (omega = (0, wy, wz), so x is constant)
    if (xs < P.bx0 || xs > P.bx1) ok = false;
    if (wy != 0.0) {
      double t1 = (P.by0 - P0y) * P.inv_wy, t2 = (P.by1 - P0y) * P.inv_wy;
      lo = fmax(lo, fmin(t1, t2));
      hi = fmin(hi, fmax(t1, t2));
    } else if (P0y < P.by0 || P0y > P.by1) {
      ok = false;
    }
    if (wz != 0.0) {
      double t1 = (P.bz0 - P0z) * P.inv_wz, t2 = (P.bz1 - P0z) * P.inv_wz;
      lo = fmax(lo, fmin(t1, t2));
      hi = fmin(hi, fmax(t1, t2));
    } else if (P0z < P.bz0 || P0z > P.bz1) {
      ok = false;
    }
  } else if (wz != 0.0) {
    double t1 = (-P.H_cyl - P0z) * P.inv_wz, t2 = (P.H_cyl - P0z) * P.inv_wz;
    lo = fmax(lo, fmin(t1, t2));
    hi = fmin(hi, fmax(t1, t2));
  } else if (fabs(P0z) > P.H_cyl) {
    ok = false;
  }
  double c = xs * xs + P0y * P0y - P.R_cyl * P.R_cyl;
  if (P.box || P.sph) {
    // (the box or sphere chord is complete)
  } else if (wy != 0.0) {
    // roots of a s^2 + b s + c with a = wy^2, b = 2 P0y wy: (-b -+ sqrt(b^2 - 4 a c)) / (2 a),
    // the discriminant as 4 a (R - x)(R + x) (equal: x is constant along the ray; the
    // difference of squares would lose the chords of grazing rays)
    double b = 2.0 * P0y * wy;
    double disc = 4.0 * (wy * wy) * ((P.R_cyl - xs) * (P.R_cyl + xs));
    if (disc < 0.0) {
      ok = false;
    } else {
      double sq = sqrt(disc);
      lo = fmax(lo, (-b - sq) * P.inv_2a);
      hi = fmin(hi, (-b + sq) * P.inv_2a);
    }
  } else if (c > 0.0) {
    ok = false;
  }
  ok = ok && (hi > lo);
  if (!ok) {
    lo = 0.0;
    hi = 0.0;
  }
  double ds = (hi - lo) * P.inv_ns;
  double s0 = lo + 0.5 * ds;
  double yb = P0y + s0 * wy, zb = P0z + s0 * wz, dy = ds * wy, dz = ds * wz;
  R.x = (float)xs;
  R.yb = (float)yb;
  R.yb2 = (float)(yb - (double)R.yb);
  R.zb = (float)zb;
  R.zb2 = (float)(zb - (double)R.zb);
  double dyh = round_bits(dy, P.step_bits), dzh = round_bits(dz, P.step_bits);
  R.dy = (float)dyh;
  R.dy2 = (float)(dy - dyh);
  R.dz = (float)dzh;
  R.dz2 = (float)(dz - dzh);
  R.ds = (float)ds;
  R.vfac = (float)((double)P.vk * P.sin_i * xs);
  R.hit = ok ? 1 : 0;
  R.pix = iy * P.nx + ix;
  R.klo = 0;
  R.khi = ok ? P.n_samples - 1 : -1;
  if (ok && !P.box && !P.sph && !P.full_range)
    gas_range(P, (float)xs, (float)P0y, (float)P0z, (float)wy, (float)wz, (float)lo, (float)hi,
              &R.klo, &R.khi);
  return R;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Field lookup state, also used by the adjoint to scatter gradients.
struct Cell {
  int i0, j0;
  float fr, fz;
  float zr;
  float ir;  // 1 / r
  bool gas;
};

// Gas is inside the grid: r >= r_in and |z|/r <= zr_max (as z^2 <= zr_max^2 r^2).
__device__ __forceinline__ bool in_gas(const MarchParams &P, float z, float r2) {
  return (r2 >= P.r_in2) && (z * z <= P.zr_max2 * r2);
}

// LOG: the radial grid is known to be log-spaced (specialised kernels).
template <bool LOG = false>
__device__ __forceinline__ Cell locate(const MarchParams &P, float z, float r2) {
  Cell c;
  float ir = rsq(r2);
  float zr = fabsf(z) * ir;
  c.gas = in_gas(P, z, r2);
  float u = (LOG || P.r_log) ? lg2(r2 * P.inv_rin2) * P.lr_scale
                             : fmaf(r2 * ir, P.lr_scale, P.lr_off);
  u = fminf(fmaxf(u, 0.0f), (float)(P.nr - 1));
  int i0 = min((int)u, P.nr - 2);
  float w = fminf(fmaxf(zr * P.w_scale, 0.0f), (float)(P.nz - 1));
  int j0 = min((int)w, P.nz - 2);
  c.i0 = i0;
  c.j0 = j0;
  c.fr = u - (float)i0;
  c.fz = w - (float)j0;
  c.zr = zr;
  c.ir = ir;
  return c;
}

__device__ __forceinline__ float bilerp(const float *__restrict__ F, int nr, const Cell &c) {
  const float *p = F + c.j0 * nr + c.i0;
  float f00 = __ldg(p), f01 = __ldg(p + 1), f10 = __ldg(p + nr), f11 = __ldg(p + nr + 1);
  return lerpf(lerpf(f00, f01, c.fr), lerpf(f10, f11, c.fr), c.fz);
}

__device__ __forceinline__ float quad_lerp(const float4 &q, const Cell &c) {
  return lerpf(lerpf(q.x, q.y, c.fr), lerpf(q.z, q.w, c.fr), c.fz);
}

// Interpolated node fields at a located sample (the arithmetic of bilerp either way).
struct NodeVals {
  float T, n, vt, hlo, hhi;
  float vphi;  // rotation field (only with P.vphi)
};

// ROT: the problem has a rotation field (then the corner quads hold four fields per cell,
// otherwise three). QUADS: the corner quads are known to be packed (specialised kernels).
template <bool ROT, bool QUADS = false>
__device__ __forceinline__ NodeVals fields_at(const MarchParams &P, const Cell &c) {
  NodeVals v;
  if (QUADS || P.cell) {
    const float4 *q = P.cell + (ROT ? 4 : 3) * ((long long)c.j0 * (P.nr - 1) + c.i0);
    const float4 qT = __ldg(q), qn = __ldg(q + 1), qv = __ldg(q + 2);
    v.vphi = ROT ? quad_lerp(__ldg(q + 3), c) : 0.0f;
    const float4 qh = __ldg(P.hcell + c.i0);
    v.T = quad_lerp(qT, c);
    v.n = quad_lerp(qn, c);
    v.vt = quad_lerp(qv, c);
    v.hlo = lerpf(qh.x, qh.y, c.fr);
    v.hhi = lerpf(qh.z, qh.w, c.fr);
  } else {
    v.T = bilerp(P.T, P.nr, c);
    v.n = bilerp(P.n, P.nr, c);
    v.vt = bilerp(P.vt, P.nr, c);
    v.vphi = ROT ? bilerp(P.vphi, P.nr, c) : 0.0f;
    const float *hl = P.hlo + c.i0;
    const float *hh = P.hhi + c.i0;
    v.hlo = lerpf(__ldg(hl), __ldg(hl + 1), c.fr);
    v.hhi = lerpf(__ldg(hh), __ldg(hh + 1), c.fr);
  }
  return v;
}

// Keplerian factor (r^2 + z^2)^{-3/4} with a refined reciprocal square root (the profile
// argument scales the relative error of v_los by v_los / alpha).
__device__ __forceinline__ float kepler_q(float d2) {
  float q = rsq(d2);
  q = q * fmaf(-0.5f * d2 * q, q, 1.5f);  // one Newton step
  return q * sqa(q);
}

// Hermite table evaluation: returns Phi and (optionally) dPhi/dt per unit t = log2 T.
__device__ __forceinline__ float lte_phi(const float *__restrict__ tab, float t, float *dphi) {
  float xt = (t - kTabT0) * kTabInvH;
  xt = fminf(fmaxf(xt, 0.0f), (float)kTabSeg);
  int i = min((int)xt, kTabSeg - 1);
  float f = xt - (float)i;
  float4 c = reinterpret_cast<const float4 *>(tab)[i];
  if (dphi) *dphi = fmaf(f, fmaf(f, 3.0f * c.w, 2.0f * c.z), c.y) * kTabInvH;
  return fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
}

// Line physics of a sample from its primitives: thermal + turbulent width, LTE source and
// tabulated opacity factor; returns {kd, a, b, S} (see sample_physics). ABS: the turbulence is
// known to be absolute (km/s, not a Mach number; specialised kernels).
template <bool ABS = false>
__device__ __forceinline__ float4 line_tail(const MarchParams &P, const float *tab, float T,
                                            float n, float X, float vt, float vlos, float ds) {
  float4 out;
  // line width
  float Tg = fmaxf(T, 1e-3f);
  float a2 = (!ABS && P.vturb_mach) ? Tg * fmaf(P.c_mach, vt * vt, P.c_th)
                                    : fmaf(P.c_th, Tg, vt * vt);
  float ia = rsq(a2);
  // LTE: source function and tabulated lower-level opacity factor
  float phi = lte_phi(tab, lg2(Tg), nullptr);
  float eS = ex2(-P.theta_s * rcp(Tg));
  out.w = eS * rcp(1.0f - eS);
  out.x = P.kappa_k * (X * n) * ex2(phi) * ia * ds;
  out.z = ia * 1.2011224087864498f;  // b = sqrt(log2 e) / alpha
  out.y = vlos * out.z;              // a = v_los b
  return out;
}

// Channel-independent physics of sample k of a ray: {kd, a, b, S} with
//   kd  optical depth per unit profile (log2 units): dtau_c = kd 2^{-d_c^2}, 0 without gas
//   a,b profile argument d_c = v_c b - a (b = sqrt(log2 e)/alpha, a = v_los b)
//   S   LTE source function in units of 2 h nu0^3 / c^2
// SPEC: the common configuration is known at compile time (spec_ok: packed corner quads, log
// radial grid, logistic CO edges, absolute turbulence, no network modulation), so its
// branches on the parameters are removed.
template <bool ROT = false, bool SPEC = false>
__device__ __forceinline__ float4 sample_physics(const MarchParams &P, const float *tab,
                                                 const Ray &R, int k) {
  float kf = (float)k;
  float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  float r2 = fmaf(R.x, R.x, y * y);
  // samples without gas leave before the grid location (two multiplies and compares)
  if (!(in_gas(P, z, r2) && k <= R.khi)) return make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  Cell c = locate<SPEC>(P, z, r2);
  const NodeVals f = fields_at<ROT, SPEC>(P, c);
  float T = f.T, n = f.n, vt = f.vt, hlo = f.hlo, hhi = f.hhi;
  if (!SPEC && P.mod) {
    const float4 o = __ldg(P.mod + (long long)R.pix * P.n_samples + k);
    T *= ex2(o.x * 1.4426950408889634f);
    n *= ex2(o.y * 1.4426950408889634f);
    hlo = fmaf(P.h_scale, o.z, hlo);
    hhi = fmaf(P.h_scale, o.w, hhi);
  }
  float X;
  if (!SPEC && P.hard_edge) {
    X = (c.zr >= hlo && c.zr <= hhi) ? P.x_co : 0.0f;
  } else {
    float ea = ex2((hlo - c.zr) * P.edge_k);
    float eb = ex2((c.zr - hhi) * P.edge_k);
    X = P.x_co * rcp((1.0f + ea) * (1.0f + eb));
  }
  // Keplerian rotation: v_los = sqrt(GM) sin i x (r^2 + z^2)^{-3/4} + v_sys
  float vlos = ROT ? fmaf(f.vphi * (P.sin_if * R.x), c.ir, P.vsys)
                  : fmaf(R.vfac, kepler_q(fmaf(z, z, r2)), P.vsys);
  return line_tail<SPEC>(P, tab, T, n, X, vt, vlos, R.ds);
}

// The configuration the specialised kernels assume (see sample_physics).
__host__ __device__ inline bool spec_ok(const MarchParams &P) {
  return P.cell != nullptr && P.r_log && !P.hard_edge && !P.vturb_mach && P.mod == nullptr &&
         P.v_uniform && P.dv != 0.0f && !P.no_window && !P.box && !P.sph;
}

// Two-lane FP32 arithmetic (FFMA2 / FMUL2 / FADD2: one instruction for two independent
// operations, each rounded as its scalar form).
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 t) {
  return __ffma2_rn(t, sub2(b, a), a);
}

// sample_physics<ROT, true> for two samples k0, k1 of one ray at once: the same operations in
// the same order, the FP32 ones issued as two-lane instructions (the MUFU operations, the
// clamps and the loads stay per sample), so each result is bit-identical to the scalar
// form's. Both samples are evaluated when either has gas (the grid location clamps the cell
// indices, so a sample without gas reads valid cells); a sample without gas returns
// {0, 0, 1, 0}.
template <bool ROT>
__device__ __forceinline__ void sample_physics_x2(const MarchParams &P, const float *tab,
                                                  const Ray &R, int k0, int k1, float4 &o0,
                                                  float4 &o1) {
  const float2 kf = make_float2((float)k0, (float)k1);
  const float2 y = __fadd2_rn(__ffma2_rn(kf, bc2(R.dy), bc2(R.yb)),
                              __ffma2_rn(kf, bc2(R.dy2), bc2(R.yb2)));
  const float2 z = __fadd2_rn(__ffma2_rn(kf, bc2(R.dz), bc2(R.zb)),
                              __ffma2_rn(kf, bc2(R.dz2), bc2(R.zb2)));
  const float2 r2 = __ffma2_rn(bc2(R.x), bc2(R.x), __fmul2_rn(y, y));
  const float2 zz = __fmul2_rn(z, z), lim = __fmul2_rn(bc2(P.zr_max2), r2);
  const bool g0 = (r2.x >= P.r_in2) && (zz.x <= lim.x) && k0 <= R.khi;
  const bool g1 = (r2.y >= P.r_in2) && (zz.y <= lim.y) && k1 <= R.khi;
  o0 = o1 = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  if (!(g0 || g1)) return;
  // grid location (locate<true>)
  const float2 ir = make_float2(rsq(r2.x), rsq(r2.y));
  const float2 zr = __fmul2_rn(make_float2(fabsf(z.x), fabsf(z.y)), ir);
  const float2 lr = __fmul2_rn(r2, bc2(P.inv_rin2));
  float2 u = __fmul2_rn(make_float2(lg2(lr.x), lg2(lr.y)), bc2(P.lr_scale));
  float2 w = __fmul2_rn(zr, bc2(P.w_scale));
  const float umax = (float)(P.nr - 1), wmax = (float)(P.nz - 1);
  u = make_float2(fminf(fmaxf(u.x, 0.0f), umax), fminf(fmaxf(u.y, 0.0f), umax));
  w = make_float2(fminf(fmaxf(w.x, 0.0f), wmax), fminf(fmaxf(w.y, 0.0f), wmax));
  const int ia0 = min((int)u.x, P.nr - 2), ia1 = min((int)u.y, P.nr - 2);
  const int ja0 = min((int)w.x, P.nz - 2), ja1 = min((int)w.y, P.nz - 2);
  const float2 fr = __fadd2_rn(u, make_float2(-(float)ia0, -(float)ia1));
  const float2 fz = __fadd2_rn(w, make_float2(-(float)ja0, -(float)ja1));
  // corner quads (fields_at<ROT, true>)
  constexpr int NQ = ROT ? 4 : 3;
  const float4 *qa = P.cell + NQ * ((long long)ja0 * (P.nr - 1) + ia0);
  const float4 *qb = P.cell + NQ * ((long long)ja1 * (P.nr - 1) + ia1);
  const float4 aT = __ldg(qa), an = __ldg(qa + 1), av = __ldg(qa + 2);
  const float4 bT = __ldg(qb), bn = __ldg(qb + 1), bv = __ldg(qb + 2);
  const float4 ah = __ldg(P.hcell + ia0), bh = __ldg(P.hcell + ia1);
  auto qlerp = [&](const float4 &a, const float4 &b) {
    const float2 lo = lerp2(make_float2(a.x, b.x), make_float2(a.y, b.y), fr);
    const float2 hi = lerp2(make_float2(a.z, b.z), make_float2(a.w, b.w), fr);
    return lerp2(lo, hi, fz);
  };
  const float2 T = qlerp(aT, bT), n = qlerp(an, bn), vt = qlerp(av, bv);
  const float2 hlo = lerp2(make_float2(ah.x, bh.x), make_float2(ah.y, bh.y), fr);
  const float2 hhi = lerp2(make_float2(ah.z, bh.z), make_float2(ah.w, bh.w), fr);
  // logistic CO edges
  const float2 xa = __fmul2_rn(sub2(hlo, zr), bc2(P.edge_k));
  const float2 xb = __fmul2_rn(sub2(zr, hhi), bc2(P.edge_k));
  const float2 ea = make_float2(ex2(xa.x), ex2(xa.y)), eb = make_float2(ex2(xb.x), ex2(xb.y));
  const float2 den = __fmul2_rn(__fadd2_rn(bc2(1.0f), ea), __fadd2_rn(bc2(1.0f), eb));
  const float2 X = __fmul2_rn(bc2(P.x_co), make_float2(rcp(den.x), rcp(den.y)));
  // line-of-sight velocity
  float2 vlos;
  if (ROT) {
    const float2 vp = qlerp(__ldg(qa + 3), __ldg(qb + 3));
    vlos = __ffma2_rn(__fmul2_rn(vp, bc2(P.sin_if * R.x)), ir, bc2(P.vsys));
  } else {
    const float2 d2 = __ffma2_rn(z, z, r2);
    float2 kq = make_float2(rsq(d2.x), rsq(d2.y));
    const float2 h = __fmul2_rn(__fmul2_rn(bc2(-0.5f), d2), kq);
    kq = __fmul2_rn(kq, __ffma2_rn(h, kq, bc2(1.5f)));
    kq = __fmul2_rn(kq, make_float2(sqa(kq.x), sqa(kq.y)));
    vlos = __ffma2_rn(bc2(R.vfac), kq, bc2(P.vsys));
  }
  // line physics (line_tail<true>)
  const float2 Tg = make_float2(fmaxf(T.x, 1e-3f), fmaxf(T.y, 1e-3f));
  const float2 a2 = __ffma2_rn(bc2(P.c_th), Tg, __fmul2_rn(vt, vt));
  const float2 ia = make_float2(rsq(a2.x), rsq(a2.y));
  float2 xt = __fmul2_rn(make_float2(lg2(Tg.x), lg2(Tg.y)), bc2(kTabInvH));
  xt = make_float2(fminf(fmaxf(xt.x, 0.0f), (float)kTabSeg),
                   fminf(fmaxf(xt.y, 0.0f), (float)kTabSeg));
  const int ta = min((int)xt.x, kTabSeg - 1), tb = min((int)xt.y, kTabSeg - 1);
  const float2 f = __fadd2_rn(xt, make_float2(-(float)ta, -(float)tb));
  const float4 ca = reinterpret_cast<const float4 *>(tab)[ta];
  const float4 cb = reinterpret_cast<const float4 *>(tab)[tb];
  float2 phi = __ffma2_rn(f, make_float2(ca.w, cb.w), make_float2(ca.z, cb.z));
  phi = __ffma2_rn(f, phi, make_float2(ca.y, cb.y));
  phi = __ffma2_rn(f, phi, make_float2(ca.x, cb.x));
  const float2 es = __fmul2_rn(bc2(-P.theta_s), make_float2(rcp(Tg.x), rcp(Tg.y)));
  const float2 eS = make_float2(ex2(es.x), ex2(es.y));
  const float2 om = __fadd2_rn(bc2(1.0f), neg2(eS));
  const float2 S = __fmul2_rn(eS, make_float2(rcp(om.x), rcp(om.y)));
  float2 kd = __fmul2_rn(bc2(P.kappa_k), __fmul2_rn(X, n));
  kd = __fmul2_rn(__fmul2_rn(__fmul2_rn(kd, make_float2(ex2(phi.x), ex2(phi.y))), ia),
                  bc2(R.ds));
  const float2 b = __fmul2_rn(ia, bc2(1.2011224087864498f));
  const float2 a = __fmul2_rn(vlos, b);
  if (g0) o0 = make_float4(kd.x, a.x, b.x, S.x);
  if (g1) o1 = make_float4(kd.y, a.y, b.y, S.y);
}

// Sample physics on a 3-D Cartesian grid (rt_render3d): trilinear interpolation of the
// packed node records {T, n, vt, x_co} and {vx, vy, vz, 0} (16 loads of 16 bytes), the
// line-of-sight velocity omega . v + v_sys with omega = (0, sin i, -cos i), then the line
// physics of every mode. No gas outside the box.
__device__ __forceinline__ float4 sample_physics_box(const MarchParams &P, const float *tab,
                                                     const Ray &R, int k) {
  const float kf = (float)k;
  const float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  const float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  float4 out = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  if (!(k <= R.khi)) return out;
  // cell index and weight per axis, from the offset to the axis' central node
  auto axis = [](float pos, float c, float s, int k, int n, int &i, float &w) {
    const float f = (pos - c) * s;
    const float fl = floorf(f);
    i = k + (int)fl;
    w = f - fl;
    if (i < 0) {
      i = 0;
      w = 0.0f;
    } else if (i > n - 2) {
      i = n - 2;
      w = 1.0f;
    }
  };
  int ix, iy, iz;
  float wx, wy, wz;
  axis(R.x, P.g3cx, P.g3sx, P.g3kx, P.n3x, ix, wx);
  axis(y, P.g3cy, P.g3sy, P.g3ky, P.n3y, iy, wy);
  axis(z, P.g3cz, P.g3sz, P.g3kz, P.n3z, iz, wz);
  const long long sy = P.n3x, sz = (long long)P.n3x * P.n3y;
  const long long b = iz * sz + iy * sy + ix;
  const long long o[8] = {b, b + 1, b + sy, b + sy + 1, b + sz, b + sz + 1, b + sz + sy,
                          b + sz + sy + 1};
  float4 a[8], v[8];
#pragma unroll
  for (int c = 0; c < 8; c++) {
    a[c] = __ldg(P.node_a + o[c]);
    v[c] = __ldg(P.node_b + o[c]);
  }
  // trilinear: along x, then y, then z
  auto tri = [&](float f0, float f1, float f2, float f3, float f4, float f5, float f6, float f7) {
    const float x0 = lerpf(f0, f1, wx), x1 = lerpf(f2, f3, wx);
    const float x2 = lerpf(f4, f5, wx), x3 = lerpf(f6, f7, wx);
    return lerpf(lerpf(x0, x1, wy), lerpf(x2, x3, wy), wz);
  };
  const float T = tri(a[0].x, a[1].x, a[2].x, a[3].x, a[4].x, a[5].x, a[6].x, a[7].x);
  const float n = tri(a[0].y, a[1].y, a[2].y, a[3].y, a[4].y, a[5].y, a[6].y, a[7].y);
  const float vt = tri(a[0].z, a[1].z, a[2].z, a[3].z, a[4].z, a[5].z, a[6].z, a[7].z);
  const float X = tri(a[0].w, a[1].w, a[2].w, a[3].w, a[4].w, a[5].w, a[6].w, a[7].w);
  const float vy = tri(v[0].y, v[1].y, v[2].y, v[3].y, v[4].y, v[5].y, v[6].y, v[7].y);
  const float vz = tri(v[0].z, v[1].z, v[2].z, v[3].z, v[4].z, v[5].z, v[6].z, v[7].z);
  if (!(X * n > 0.0f)) return out;
  const float vlos = fmaf(P.sin_if, vy, fmaf(-P.cos_if, vz, P.vsys));
  return line_tail(P, tab, T, n, X, vt, vlos, R.ds);
}

// Sample physics on a 3-D spherical grid (rt_render_sph): (r, theta, phi) of the sample
// (theta = atan2(R, z) from +z with R = sqrt(x^2 + y^2), phi = atan2(y, x) in [0, 2 pi)),
// trilinear interpolation of the packed node records in (radial index, theta, phi), periodic
// in phi (16 loads of 16 bytes), and v_los = omega . v + v_sys for
// v = v_r r^ + v_theta theta^ + v_phi phi^, omega = (0, sin i, -cos i):
//   v_y = (v_r sin th + v_theta cos th) sin ph + v_phi cos ph,  v_z = v_r cos th - v_theta sin th.
// No gas outside r_in <= r <= r_out, th0 <= theta <= th1. On the axis theta^ and phi^ are
// taken as 0, at the centre r^ as well.
__device__ __forceinline__ float4 sample_physics_sph(const MarchParams &P, const float *tab,
                                                     const Ray &R, int k) {
  const float kf = (float)k;
  const float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  const float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  float4 out = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  if (!(k <= R.khi)) return out;
  const float Rc2 = fmaf(R.x, R.x, y * y);
  const float r2 = fmaf(z, z, Rc2);
  if (!(r2 >= P.r_in2 && r2 <= P.r_out2)) return out;
  const float iRc = Rc2 > 0.0f ? rsq(Rc2) : 0.0f;
  const float Rc = Rc2 * iRc;
  const float th = atan2f(Rc, z);
  if (!(th >= P.th0 && th <= P.th1)) return out;
  float ph = atan2f(y, R.x);
  if (ph < 0.0f) ph += 6.283185307179586f;
  const float ir = r2 > 0.0f ? rsq(r2) : 0.0f;  // r^ taken as 0 at the centre
  float u = P.r_log ? lg2(r2 * P.inv_rin2) * P.lr_scale : fmaf(r2 * ir, P.lr_scale, P.lr_off);
  u = fminf(fmaxf(u, 0.0f), (float)(P.snr - 1));
  const int i0 = min((int)u, P.snr - 2);
  const float fr = u - (float)i0;
  const float v = fminf(fmaxf((th - P.th0) * P.th_scale, 0.0f), (float)(P.snth - 1));
  const int j0 = min((int)v, P.snth - 2);
  const float ft = v - (float)j0;
  const float w = ph * P.ph_scale;
  int k0 = (int)w;
  const float fp = w - (float)k0;
  if (k0 >= P.snph) k0 -= P.snph;  // phi rounded up to 2 pi
  const int k1 = k0 + 1 == P.snph ? 0 : k0 + 1;
  const long long sj = P.snr, sk0 = (long long)k0 * P.snth * P.snr,
                  sk1 = (long long)k1 * P.snth * P.snr;
  const long long b0 = sk0 + j0 * sj + i0, b1 = sk1 + j0 * sj + i0;
  const long long o[8] = {b0, b0 + 1, b0 + sj, b0 + sj + 1, b1, b1 + 1, b1 + sj, b1 + sj + 1};
  float4 a[8], vv[8];
#pragma unroll
  for (int c = 0; c < 8; c++) {
    a[c] = __ldg(P.node_a + o[c]);
    vv[c] = __ldg(P.node_b + o[c]);
  }
  // trilinear: along r, then theta, then phi
  auto tri = [&](float f0, float f1, float f2, float f3, float f4, float f5, float f6, float f7) {
    const float x0 = lerpf(f0, f1, fr), x1 = lerpf(f2, f3, fr);
    const float x2 = lerpf(f4, f5, fr), x3 = lerpf(f6, f7, fr);
    return lerpf(lerpf(x0, x1, ft), lerpf(x2, x3, ft), fp);
  };
  const float T = tri(a[0].x, a[1].x, a[2].x, a[3].x, a[4].x, a[5].x, a[6].x, a[7].x);
  const float n = tri(a[0].y, a[1].y, a[2].y, a[3].y, a[4].y, a[5].y, a[6].y, a[7].y);
  const float vt = tri(a[0].z, a[1].z, a[2].z, a[3].z, a[4].z, a[5].z, a[6].z, a[7].z);
  const float X = tri(a[0].w, a[1].w, a[2].w, a[3].w, a[4].w, a[5].w, a[6].w, a[7].w);
  if (!(X * n > 0.0f)) return out;
  const float vr = tri(vv[0].x, vv[1].x, vv[2].x, vv[3].x, vv[4].x, vv[5].x, vv[6].x, vv[7].x);
  const float vth = tri(vv[0].y, vv[1].y, vv[2].y, vv[3].y, vv[4].y, vv[5].y, vv[6].y, vv[7].y);
  const float vph = tri(vv[0].z, vv[1].z, vv[2].z, vv[3].z, vv[4].z, vv[5].z, vv[6].z, vv[7].z);
  const float sth = Rc * ir, cth = z * ir;                  // sin, cos theta
  const float sph_ = y * iRc, cph = R.x * iRc;              // sin, cos phi (0 on the axis)
  const float vy = fmaf(fmaf(vr, sth, vth * cth), sph_, vph * cph);
  const float vz = fmaf(vr, cth, -vth * sth);
  const float vlos = fmaf(P.sin_if, vy, fmaf(-P.cos_if, vz, P.vsys));
  return line_tail(P, tab, T, n, X, vt, vlos, R.ds);
}

// Sample physics of the forward march by mode: 0 axisymmetric grid, Keplerian rotation; 1
// axisymmetric grid with a rotation field; 2 3-D Cartesian grid; 3 3-D spherical grid; 4 and 5
// modes 0 and 1 specialised for the common configuration (spec_ok).
template <int MODE>
__device__ __forceinline__ float4 march_physics(const MarchParams &P, const float *tab,
                                                const Ray &R, int k) {
  if (MODE == 3) return sample_physics_sph(P, tab, R, k);
  if (MODE == 2) return sample_physics_box(P, tab, R, k);
  if (MODE >= 4) return sample_physics<MODE == 5, true>(P, tab, R, k);
  return sample_physics<MODE == 1>(P, tab, R, k);
}

// Host-side helpers (rt_api.cu, rt_forward.cu, rt_adjoint.cu)
int build_params(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                 const rt_view *view, const rt_line *line, MarchParams *P);
int set_error(int code, const char *fmt, ...);
void clear_error();
int launch_forward(const MarchParams &P, float *cube, cudaStream_t stream);
int launch_forward_dense(const MarchParams &P, float *cube, cudaStream_t stream);
int launch_plain(const MarchParams &P, float *cube, cudaStream_t stream);  // rt_plain.cu
// Stream-ordered allocation from a library-owned pool of the current device, which keeps up
// to kPoolKeepBytes cached between calls (so repeated renders do not map and unmap their
// scratch); free with cudaFreeAsync.
constexpr unsigned long long kPoolKeepBytes = 1ull << 30;
cudaError_t stream_alloc(void **p, size_t bytes, cudaStream_t stream);
size_t cell_bytes(const MarchParams &P);
int launch_pressure_vphi(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                         const float *n, const float *T, float *vphi, cudaStream_t stream);
int launch_pressure_vphi_adjoint(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                                 const float *n, const float *T, const double *g_v, double *g_n,
                                 double *g_T, cudaStream_t stream);
int launch_field_chain(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                       const rt_chain &c, const float *T, float *n, float *N, float *h_lo,
                       float *h_hi, cudaStream_t stream);
int launch_field_chain_adjoint(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                               const rt_chain &c, const float *T, const double *g_n,
                               const double *g_lo, const double *g_hi, double *g_T,
                               cudaStream_t stream);
int pack_cells(MarchParams &P, void *buf, cudaStream_t stream);
int launch_count(const MarchParams &P, unsigned long long *count, cudaStream_t stream);
void lane_layout(int nch, bool dense, int *lpr, int *cpl);
int launch_adjoint(const MarchParams &P, const float *dLdc, const float *target, float *cube_out,
                   const rt_grads &G, cudaStream_t stream, float4 *dmod = nullptr,
                   unsigned *dmax = nullptr);
void adj_layout(int nch, int *lpr, int *cpl);
// the fused adjoint on a 3-D grid (P.box or P.sph, with its node records packed)
int launch_adjoint3(const MarchParams &P, const float *dLdc, const float *target,
                    float *cube_out, const rt_grads3 &G3, cudaStream_t stream);
size_t adjoint_scratch_bytes(const MarchParams &P, long long cap_blocks);
int check_adjoint_args(const MarchParams &P, const float *dL_dcube, const float *target,
                       const rt_grads *grads);
int launch_mlp_rays(const rt_mlp *m, const MarchParams &P, float4 *mod, void *ray_buf,
                    void *list_buf, cudaStream_t stream);
size_t ray_buffer_bytes(long long npix);
// ray setups of every pixel of P into rays (ray_buffer_bytes(nx ny) bytes)
int launch_rays(const MarchParams &P, Ray *rays, cudaStream_t stream);
size_t sample_list_bytes(long long npix, int n_samples);
int mlp_validate(const rt_mlp *m);
int mlp_grads_validate(const rt_mlp_grads *g);
size_t mlp_bwd_scratch_bytes(long long n);
// entries of the gathered backward inputs (xy and g buffers) for n samples
size_t mlp_bwd_gather_entries(long long n);
int launch_mlp_bwd_rays(const rt_mlp *m, const MarchParams &P, const void *ray_buf,
                        const void *list_buf, const float4 *dmod, const unsigned *dmax,
                        void *spill, float2 *xy_buf, float4 *g_buf, const rt_mlp_grads *g,
                        cudaStream_t stream);
int launch_coords(const MarchParams &P, float2 *xy, cudaStream_t stream);
int launch_surface_grad(const rt_grid &g, const double *dh, const float *h, double c,
                        double *out, cudaStream_t stream);
int resident_blocks(const void *kernel, int threads);

}  // namespace rtb
