// Fused adjoint of the march: a forward march that renders the cube, forms the loss seed and
// keeps the optical depth at every batch boundary, then a reverse march that propagates
// dL/dcube back to every node of the (r, z/r) fields and the CO surfaces (and, for
// neural-field renders, to the per-sample network outputs).
//
// Gradient of one channel. With T_k = 2^-tau_k the transmittance in front of sample k,
// dt_k its optical depth (log2 units), S_k its source and S_N the background, the intensity
// is I = sum_k S_k (T_k - T_{k+1}) + S_N T_N, and
//   dI/dS_k  = T_k - T_{k+1}
//   dI/ddt_k = -ln2 A_k,   A_k = sum_{m>k} (S_m - S_{m-1}) T_m = A_{k+1} + (S_{k+1} - S_k) T_{k+1}.
// A is a suffix sum, accumulated back to front from small terms (it vanishes behind optically
// thick gas, where a front-to-back form I - prefix would leave rounding noise of order I).
// Samples without gas (dt = 0 in every channel) drop out exactly, so they are skipped and
// S_{k+1} means the source of the next sample with gas.
//
// The transmittance of the reverse march comes from optical depths summed front to back: for
// every batch of LPR samples the forward pass keeps, in the warp's scratch, the (compensated)
// optical depths at the batch's end of the channel pairs the batch advanced (the others did
// not change), and the batch's pair mask; the reverse reloads those at each batch and
// rebuilds the depths inside it by subtracting its own increments (recomputed with the
// forward pass's roundings), so no rounding carries from one batch into the next.
//
// Per sample, lane q of a ray computes the channel-independent physics of its sample with
// the local partial derivatives (kept in shared memory); the per-channel sums
//   ax = sum_c gI_c A_c g_c,  ay = sum_c gI_c A_c g_c d_c^2,  aS = sum_c gI_c (T_k - T_{k+1})
// (g_c = 2^-d_c^2 the profile, gI_c = dL/dI_c) are reduced over the lanes of the ray through
// shared memory, and lane q applies the chain rule through the line width, the LTE table,
// the Planck source, the CO-layer edges and the bilinear weights, scattering the node
// gradients with FP64 atomics into replicated accumulators.
#include <mutex>
#include <new>
#include <type_traits>

#include "rt_internal.cuh"

namespace rtb {

// warps per block: 4, or 2 where the per-warp shared memory is large (16 or 32 lanes per ray)
template <int LPR>
constexpr int adj_wpb() {
  return LPR >= 16 ? 2 : 4;
}

// Per-sample record of the batch being reversed (shared memory, one per lane): the physics
// {kd, a, b, S} and the local derivatives (below), five float4 per lane; without a network or a rotation field
// the fifth (J_MN, J_T, J_N, J_VPX: the network factor on n, the modulated primitives and
// d v_los / d v_phi) is neither written nor read.
constexpr int kRec = 5;

// Per-warp scratch in floats, for rays of nbat batches of LPR samples at most: the optical
// depths of the lanes' CPL channel slots at the end of the rays ([lane][CPL], float4 per
// lane), then one entry per (batch, channel pair the batch advances): the pair's depths at the
// end of the batch ([entry][lane] float2; nbat CPL / 2 entries at most, about a third of that
// with the channel window), then the forward pass's pair mask of every batch (one byte each).
// Only what the rays use is touched, which keeps the warps' scratch in L2.
template <int LPR, int CPL>
__host__ __device__ constexpr long long adj_warp_floats(int nbat) {
  return (long long)CPL * 32 + (long long)nbat * (CPL / 2) * 64 + (long long)(nbat + 15) / 16 * 4;
}
// Batches of LPR samples of the longest ray.
template <int LPR>
__host__ __device__ constexpr int adj_batches(int n_samples) {
  return (n_samples + LPR - 1) / LPR;
}
constexpr float kLn2 = 0.6931471805599453f;
// Cap on one sample's optical-depth increment in one channel (log2 units). Behind an increment
// of 128 the transmittance is below 2^-128, which ex2.approx.ftz returns as 0, so capping
// changes no transmittance, no intensity and no gradient term (every term behind the sample
// carries that zero). It bounds a batch's depth range by LPR x 128, so the depths the reverse
// pass rebuilds by subtracting increments from a batch end keep an absolute error of a few
// 1e-5: without it one optically very thick sample (increments of 1e5 in a dense midplane)
// left ulp(1e5) ~ 1e-2 of error in the depths in front of it. Both passes form each increment
// as the rounded product kd g, capped, so the reverse subtracts exactly what the forward added.
constexpr float kDtCap = 128.0f;

// Per-sample local derivatives kept in shared memory between the physics and the chain rule.
enum {
  J_KDN,   // kd / n
  J_DPHI,  // d ln(2^Phi) / dT = Phi'(log2 T) / T           (0 where T is clamped)
  J_QT,    // -1/2 ia^2 d(alpha^2)/dT                         (0 where T is clamped)
  J_QV,    // -1/2 ia^2 d(alpha^2)/dv_turb
  J_DS,    // dS/dT                                          (0 where T is clamped)
  J_SA,    // d ln X / d h_lo
  J_SB,    // d ln X / d h_hi
  J_FR,    // bilinear weights
  J_FZ,
  J_CELL,  // node index j0 * nr + i0 (int bits)
  J_I0,    // radial node index i0 (int bits)
  J_MT,    // network factor on T (e^{o0}; 1 for grid fields)
  J_MN,    // network factor on n (e^{o1})
  J_T,     // T and n after the network factors
  J_N,
  J_VPX,   // d v_los / d v_phi = sin i x / r (with a rotation field)
  kJ
};
static_assert(kJ <= 4 * (kRec - 1), "local derivatives fit the sample record");
static_assert(J_MN == 4 * (kRec - 2) && J_T > J_MN && J_N > J_MN && J_VPX > J_MN && J_MT < J_MN,
              "the last record slot holds the network and rotation-field entries");

// Channel-independent physics of sample k with its local derivatives, written where the sample
// has gas to the record slots rec[32 (i + 1)], i < kRec - 1 (entries 4i .. 4i + 3 of the enum).
// Returns {kd, a, b, S} as sample_physics does for a sample with gas, and zeros (b = 0 marks
// "no gas") otherwise. The arithmetic of kd, a, b and S is the same as sample_physics'.
template <bool ROT, bool SPEC = false>
__device__ __forceinline__ float4 physics_jac(const MarchParams &P, const float *tab,
                                              const Ray &R, int k, float4 *rec) {
  const float kf = (float)k;
  const float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  const float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  const float r2 = fmaf(R.x, R.x, y * y);
  if (!(in_gas(P, z, r2) && k <= R.khi)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const Cell c = locate<SPEC>(P, z, r2);
  const NodeVals f = fields_at<ROT, SPEC>(P, c);
  float T = f.T, n = f.n, hlo = f.hlo, hhi = f.hhi;
  const float vt = f.vt;
  float mT = 1.0f, mn = 1.0f;
  if (!SPEC && P.mod) {
    const float4 o = __ldg(P.mod + (long long)R.pix * P.n_samples + k);
    mT = ex2(o.x * 1.4426950408889634f);
    mn = ex2(o.y * 1.4426950408889634f);
    T *= mT;
    n *= mn;
    hlo = fmaf(P.h_scale, o.z, hlo);
    hhi = fmaf(P.h_scale, o.w, hhi);
  }
  float X, sa = 0.0f, sb = 0.0f;
  if (!SPEC && P.hard_edge) {
    X = (c.zr >= hlo && c.zr <= hhi) ? P.x_co : 0.0f;
  } else {
    // X = x_co / ((1 + ea)(1 + eb)), ea = 2^{(h_lo - z/r) k}, eb = 2^{(z/r - h_hi) k}
    const float ea = ex2((hlo - c.zr) * P.edge_k);
    const float eb = ex2((c.zr - hhi) * P.edge_k);
    const float pa = 1.0f + ea, pb = 1.0f + eb;
    const float rr = rcp(pa * pb);
    X = P.x_co * rr;
    const float kl = P.edge_k * kLn2;
    sa = -ea * pb * rr * kl;
    sb = eb * pa * rr * kl;
  }
  // v_los as in sample_physics: the rotation field projected, or the Keplerian term
  const float vpx = P.sin_if * R.x * c.ir;  // d v_los / d v_phi
  const float vlos = ROT ? fmaf(f.vphi * (P.sin_if * R.x), c.ir, P.vsys)
                         : fmaf(R.vfac, kepler_q(fmaf(z, z, r2)), P.vsys);
  const bool clampT = T < 1e-3f;
  const float Tg = fmaxf(T, 1e-3f);
  float a2, da2T, da2v;
  if (!SPEC && P.vturb_mach) {
    const float m = fmaf(P.c_mach, vt * vt, P.c_th);
    a2 = Tg * m;
    da2T = m;
    da2v = Tg * P.c_mach * 2.0f * vt;
  } else {
    a2 = fmaf(P.c_th, Tg, vt * vt);
    da2T = P.c_th;
    da2v = 2.0f * vt;
  }
  const float ia = rsq(a2);
  float dphi;
  const float phi = lte_phi(tab, lg2(Tg), &dphi);
  const float iT = rcp(Tg);
  const float eS = ex2(-P.theta_s * iT);
  const float om = rcp(1.0f - eS);
  const float F = ex2(phi);
  const float q = -0.5f * ia * ia;
  float J[4 * (kRec - 1)];
  J[J_KDN] = P.kappa_k * X * F * ia * R.ds;
  J[J_DPHI] = clampT ? 0.0f : dphi * iT;
  J[J_QT] = clampT ? 0.0f : q * da2T;
  J[J_QV] = q * da2v;
  // S = eS / (1 - eS), eS = 2^{-theta/T}: dS/dT = eS ln2 theta / (T^2 (1 - eS)^2)
  J[J_DS] = clampT ? 0.0f : eS * om * om * kLn2 * P.theta_s * iT * iT;
  J[J_SA] = sa;
  J[J_SB] = sb;
  J[J_FR] = c.fr;
  J[J_FZ] = c.fz;
  J[J_CELL] = __int_as_float(c.j0 * P.nr + c.i0);
  J[J_I0] = __int_as_float(c.i0);
  J[J_MT] = mT;
  J[J_MN] = mn;
  J[J_T] = T;
  J[J_N] = n;
  J[J_VPX] = ROT ? vpx : 0.0f;
  for (int e = kJ; e < 4 * (kRec - 1); e++) J[e] = 0.0f;
#pragma unroll
  for (int i = 0; i < kRec - 1; i++)
    if (i < kRec - 2 || (!SPEC && P.mod) || ROT)
      rec[(i + 1) * 32] = make_float4(J[4 * i], J[4 * i + 1], J[4 * i + 2], J[4 * i + 3]);
  float4 out;
  out.x = P.kappa_k * (X * n) * F * ia * R.ds;
  out.z = ia * 1.2011224087864498f;  // b = sqrt(log2 e) / alpha
  out.y = vlos * out.z;              // a = v_los b
  out.w = eS * om;
  return out;
}

// Line physics of a sample on a 3-D grid (line_tail's arithmetic, so {kd, a, b, S} are
// bit-identical to the forward march's, which the reverse pass's rebuilt depths rely on) with
// the local derivatives in physics_jac's slots where they mean the same (J_KDN, J_DPHI, J_QT,
// J_QV, J_DS) and dkd/dX in J_SA (the CO abundance is a field of its own on these grids).
__device__ __forceinline__ float4 line_jac3(const MarchParams &P, const float *tab, const Ray &R,
                                            float T, float n, float X, float vt, float vlos,
                                            float *J) {
  const bool clampT = T < 1e-3f;
  const float Tg = fmaxf(T, 1e-3f);
  float a2, da2T, da2v;
  if (P.vturb_mach) {
    const float m = fmaf(P.c_mach, vt * vt, P.c_th);
    a2 = Tg * m;
    da2T = m;
    da2v = Tg * P.c_mach * 2.0f * vt;
  } else {
    a2 = fmaf(P.c_th, Tg, vt * vt);
    da2T = P.c_th;
    da2v = 2.0f * vt;
  }
  const float ia = rsq(a2);
  float dphi;
  const float phi = lte_phi(tab, lg2(Tg), &dphi);
  const float iT = rcp(Tg);
  const float eS = ex2(-P.theta_s * iT);
  const float om = rcp(1.0f - eS);
  const float F = ex2(phi);
  const float q = -0.5f * ia * ia;
  J[J_KDN] = P.kappa_k * X * F * ia * R.ds;
  J[J_DPHI] = clampT ? 0.0f : dphi * iT;
  J[J_QT] = clampT ? 0.0f : q * da2T;
  J[J_QV] = q * da2v;
  J[J_DS] = clampT ? 0.0f : eS * om * om * kLn2 * P.theta_s * iT * iT;
  J[J_SA] = P.kappa_k * n * F * ia * R.ds;  // dkd/dX
  float4 out;
  out.x = P.kappa_k * (X * n) * F * ia * R.ds;
  out.z = ia * 1.2011224087864498f;
  out.y = vlos * out.z;
  out.w = eS * om;
  return out;
}

// Slots of the 3-D grids' records beyond line_jac3's: the cell's trilinear weights along its
// three axes, its lowest node (on the spherical grid: in the azimuth plane k0, and the node of
// the same (r, theta) in the plane k1 after it, periodic), and on the spherical grid
// d v_los / d(v_r, v_theta, v_phi) at the sample.
enum { J3_B1 = J_SB, J3_W0 = J_FR, J3_W1 = J_FZ, J3_B0 = J_CELL, J3_W2 = J_I0, J3_ER = J_MT,
       J3_ETH = 12, J3_EPH = 13 };

// physics_jac on the 3-D Cartesian grid (rt_render3d): sample_physics_box's arithmetic and
// line_jac3; zeros without gas.
__device__ __forceinline__ float4 physics_jac_box(const MarchParams &P, const float *tab,
                                                  const Ray &R, int k, float4 *rec) {
  const float kf = (float)k;
  const float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  const float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  if (!(k <= R.khi)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
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
  if (!(X * n > 0.0f)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float vlos = fmaf(P.sin_if, vy, fmaf(-P.cos_if, vz, P.vsys));
  float J[12];
  const float4 out = line_jac3(P, tab, R, T, n, X, vt, vlos, J);
  J[J3_B1] = 0.0f;
  J[J3_W0] = wx;
  J[J3_W1] = wy;
  J[J3_B0] = __int_as_float((int)b);
  J[J3_W2] = wz;
  J[J3_ER] = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; i++)
    rec[(i + 1) * 32] = make_float4(J[4 * i], J[4 * i + 1], J[4 * i + 2], J[4 * i + 3]);
  return out;
}

// physics_jac on the 3-D spherical grid (rt_render_sph): sample_physics_sph's arithmetic and
// line_jac3, the velocity factors d v_los / d(v_r, v_theta, v_phi) =
// (sin i sin th sin ph - cos i cos th, sin i cos th sin ph + cos i sin th, sin i cos ph);
// zeros without gas.
__device__ __forceinline__ float4 physics_jac_sph(const MarchParams &P, const float *tab,
                                                  const Ray &R, int k, float4 *rec) {
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float kf = (float)k;
  const float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  const float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  if (!(k <= R.khi)) return zero;
  const float Rc2 = fmaf(R.x, R.x, y * y);
  const float r2 = fmaf(z, z, Rc2);
  if (!(r2 >= P.r_in2 && r2 <= P.r_out2)) return zero;
  const float iRc = Rc2 > 0.0f ? rsq(Rc2) : 0.0f;
  const float Rc = Rc2 * iRc;
  const float th = atan2f(Rc, z);
  if (!(th >= P.th0 && th <= P.th1)) return zero;
  float ph = atan2f(y, R.x);
  if (ph < 0.0f) ph += 6.283185307179586f;
  const float ir = r2 > 0.0f ? rsq(r2) : 0.0f;
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
  if (k0 >= P.snph) k0 -= P.snph;
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
  auto tri = [&](float f0, float f1, float f2, float f3, float f4, float f5, float f6, float f7) {
    const float x0 = lerpf(f0, f1, fr), x1 = lerpf(f2, f3, fr);
    const float x2 = lerpf(f4, f5, fr), x3 = lerpf(f6, f7, fr);
    return lerpf(lerpf(x0, x1, ft), lerpf(x2, x3, ft), fp);
  };
  const float T = tri(a[0].x, a[1].x, a[2].x, a[3].x, a[4].x, a[5].x, a[6].x, a[7].x);
  const float n = tri(a[0].y, a[1].y, a[2].y, a[3].y, a[4].y, a[5].y, a[6].y, a[7].y);
  const float vt = tri(a[0].z, a[1].z, a[2].z, a[3].z, a[4].z, a[5].z, a[6].z, a[7].z);
  const float X = tri(a[0].w, a[1].w, a[2].w, a[3].w, a[4].w, a[5].w, a[6].w, a[7].w);
  if (!(X * n > 0.0f)) return zero;
  const float vr = tri(vv[0].x, vv[1].x, vv[2].x, vv[3].x, vv[4].x, vv[5].x, vv[6].x, vv[7].x);
  const float vth = tri(vv[0].y, vv[1].y, vv[2].y, vv[3].y, vv[4].y, vv[5].y, vv[6].y, vv[7].y);
  const float vph = tri(vv[0].z, vv[1].z, vv[2].z, vv[3].z, vv[4].z, vv[5].z, vv[6].z, vv[7].z);
  const float sth = Rc * ir, cth = z * ir;
  const float sph_ = y * iRc, cph = R.x * iRc;
  const float vy = fmaf(fmaf(vr, sth, vth * cth), sph_, vph * cph);
  const float vz = fmaf(vr, cth, -vth * sth);
  const float vlos = fmaf(P.sin_if, vy, fmaf(-P.cos_if, vz, P.vsys));
  float J[16];
  const float4 out = line_jac3(P, tab, R, T, n, X, vt, vlos, J);
  J[J3_B1] = __int_as_float((int)b1);
  J[J3_W0] = fr;
  J[J3_W1] = ft;
  J[J3_B0] = __int_as_float((int)b0);
  J[J3_W2] = fp;
  J[J3_ER] = fmaf(P.sin_if, sth * sph_, -P.cos_if * cth);
  J[J3_ETH] = fmaf(P.sin_if, cth * sph_, P.cos_if * sth);
  J[J3_EPH] = P.sin_if * cph;
  J[14] = J[15] = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; i++)
    rec[(i + 1) * 32] = make_float4(J[4 * i], J[4 * i + 1], J[4 * i + 2], J[4 * i + 3]);
  return out;
}

// Replicated gradient accumulators. Thousands of samples land on every node (and all samples
// of a radius on the same two surface entries), and atomics on one address are applied one
// after another; block b therefore accumulates into copy b % k and a final pass sums the
// copies in FP64 in a fixed order. A copy interleaves the node fields as float4
// {dT, dn, dvt, 0} and the surface entries as float2 {dh_lo, dh_hi}, so one sample adds to
// the grid with four 16-byte reductions and to the surfaces with two 8-byte ones (FP32 sums
// within a copy: a few hundred terms each, against 16 FP64 atomics whose FP32-to-FP64
// conversions run on the narrow FP64 pipe). g == nullptr (or h == nullptr) means the block
// adds straight into the caller's FP64 arrays.
struct GradCopies {
  float4 *g;  // kg copies of [nr * nz] {dT, dn, dvt, 0}, gstride float4 apart
  float2 *h;  // kh copies of [nr] {dh_lo, dh_hi}, hstride float2 apart
  long long gstride, hstride;
  int kg, kh;
  // 3-D grids (one copy each, the node count apart from nothing): g holds {dT, dn, dvt, dX}
  // per node, h {dL/dv_los, 0} per node on the Cartesian grid, v {dv_r, dv_theta, dv_phi, 0}
  // per node on the spherical grid
  float4 *v;
};

// Where one block's gradient contributions go.
struct GradSink {
  rt_grads G;  // caller's FP64 arrays (used where the copies below are absent)
  float4 *g;   // this block's grid copy, or nullptr
  float2 *h;   // this block's surface copy, or nullptr
  float4 *v;   // the spherical grid's velocity copy, or nullptr
};

__device__ __forceinline__ GradSink block_sink(const rt_grads &G, const GradCopies &C) {
  GradSink S;
  S.G = G;
  S.g = C.g ? C.g + (long long)(blockIdx.x % C.kg) * C.gstride : nullptr;
  S.h = C.h ? C.h + (long long)(blockIdx.x % C.kh) * C.hstride : nullptr;
  S.v = C.v;
  return S;
}

// Sums of the copies in FP64, in a fixed order:
//   grid:    dT[i], dn[i], dvt[i] = sum_c cop[c][i].{x, y, z}  (one thread per node, copy order)
//   surface: dh_lo[i], dh_hi[i]   = sum_c cop[c][i].{x, y}     (one warp per entry, below)
__global__ void sum_grid_copies_kernel(const float4 *__restrict__ cop, int k, long long stride,
                                       long long n, double *dT, double *dn, double *dvt,
                                       double *dvphi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int j = 0; j < k; j++) {
      const float4 v = cop[(long long)j * stride + i];
      a += v.x;
      b += v.y;
      c += v.z;
      d += v.w;
    }
    dT[i] = a;
    dn[i] = b;
    dvt[i] = c;
    if (dvphi) dvphi[i] = d;  // the rotation field's gradient (0 without one)
  }
}

// One warp per surface entry (there are few entries and up to 128 copies each): lane l sums
// copies l, l + 32, ... in order, then a fixed butterfly adds the lanes' partial sums, so the
// result does not depend on scheduling.
__global__ void sum_surface_copies_kernel(const float2 *__restrict__ cop, int k, long long stride,
                                          long long n, double *dlo, double *dhi) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w0; i < n; i += nw) {
    double a = 0.0, b = 0.0;
    for (int j = lane; j < k; j += 32) {
      const float2 v = cop[(long long)j * stride + i];
      a += v.x;
      b += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      dlo[i] = a;
      dhi[i] = b;
    }
  }
}

// Chain rule of one sample from the reduced channel sums (ax, ay, aS; see the file header)
// and the local derivatives J; node gradients into the block's sink, and the gradient with respect
// to the four network outputs of the sample when dmod is given (returns its largest
// magnitude, 0 otherwise).
// With a rotation field (ROT) also dL/dv_phi: d_c = v_c b - a with a = v_los b, so
// dL/dv_los = b dL/da = -2 ln2^2 kd b az, az = sum_c gI_c A_c g_c d_c, times d v_los / d v_phi.
template <bool ROT>
__device__ __forceinline__ float scatter_grad(const MarchParams &P, const float *J, float kd,
                                             float b, float ax, float ay, float az, float aS,
                                             const GradSink &G, float4 *dmod) {
  const float gx = -kLn2 * ax;                       // dL/dkd
  const float GB = 2.0f * kLn2 * kLn2 * kd * ay;     // b dL/db (a = v_los b included)
  const float gk = fmaf(gx, kd, GB);                 // alpha dL/d(1/alpha) ... times ia
  const float gT = fmaf(gx * kd, J[J_DPHI], fmaf(gk, J[J_QT], aS * J[J_DS]));
  const float gv = gk * J[J_QV];
  const float gn = gx * J[J_KDN];
  const float gl = gx * kd * J[J_SA];
  const float gh = gx * kd * J[J_SB];
  float dm = 0.0f;
  if (dmod) {
    const float4 o = make_float4(gT * J[J_T], gn * J[J_N], gl * P.h_scale, gh * P.h_scale);
    *dmod = o;
    dm = fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fmaxf(fabsf(o.z), fabsf(o.w)));
  }
  const float dT = gT * J[J_MT], dn = gn * J[J_MN];
  const float gp = ROT ? -2.0f * kLn2 * kLn2 * kd * b * az * J[J_VPX] : 0.0f;  // dL/dv_phi
  const float fr = J[J_FR], fz = J[J_FZ];
  const int i00 = __float_as_int(J[J_CELL]), i0 = __float_as_int(J[J_I0]);
  const int nr = P.nr;
  const int idx[4] = {i00, i00 + 1, i00 + nr, i00 + nr + 1};
  const float w[4] = {(1.0f - fr) * (1.0f - fz), fr * (1.0f - fz), (1.0f - fr) * fz, fr * fz};
  if (G.g) {
#pragma unroll
    for (int a = 0; a < 4; a++)
      atomicAdd(G.g + idx[a], make_float4(dT * w[a], dn * w[a], gv * w[a], gp * w[a]));
  } else {
#pragma unroll
    for (int a = 0; a < 4; a++) {
      atomicAdd(G.G.dT + idx[a], (double)(dT * w[a]));
      atomicAdd(G.G.dn + idx[a], (double)(dn * w[a]));
      atomicAdd(G.G.dvt + idx[a], (double)(gv * w[a]));
      if (ROT) atomicAdd(G.G.dvphi + idx[a], (double)(gp * w[a]));
    }
  }
  if (G.h) {
    atomicAdd(G.h + i0, make_float2(gl * (1.0f - fr), gh * (1.0f - fr)));
    atomicAdd(G.h + i0 + 1, make_float2(gl * fr, gh * fr));
  } else {
    atomicAdd(G.G.dh_lo + i0, (double)(gl * (1.0f - fr)));
    atomicAdd(G.G.dh_lo + i0 + 1, (double)(gl * fr));
    atomicAdd(G.G.dh_hi + i0, (double)(gh * (1.0f - fr)));
    atomicAdd(G.G.dh_hi + i0 + 1, (double)(gh * fr));
  }
  return dm;
}

// Chain rule of one sample on a 3-D grid (line_jac3's entries and the cell of physics_jac_box
// or physics_jac_sph): dL/d of T, n_H2, v_turb and the CO abundance as a float4 per node, and
// the velocity fields' share of dL/dv_los -- on the Cartesian grid dL/dv_los itself as the
// first entry of a float2 per node (the components' gradients are sin i and -cos i times it,
// formed when the copy is written out), on the spherical grid dL/dv_los times the sample's
// factors for v_r, v_theta, v_phi as a float4 per node -- each spread over the cell's 8 corners
// with the trilinear weights (corner bit 0 the first axis, bit 1 the second, bit 2 the third:
// z on the Cartesian grid, the next azimuth plane on the spherical one).
template <bool SPH>
__device__ __forceinline__ void scatter_3d(const MarchParams &P, const float *J, float kd,
                                           float b, float ax, float ay, float az, float aS,
                                           const GradSink &G) {
  const float gx = -kLn2 * ax;                    // dL/dkd
  const float GB = 2.0f * kLn2 * kLn2 * kd * ay;  // b dL/db
  const float gk = fmaf(gx, kd, GB);
  const float gT = fmaf(gx * kd, J[J_DPHI], fmaf(gk, J[J_QT], aS * J[J_DS]));
  const float gv = gk * J[J_QV];
  const float gn = gx * J[J_KDN];
  const float gX = gx * J[J_SA];
  const float gl = -2.0f * kLn2 * kLn2 * kd * b * az;  // dL/dv_los
  const float w0 = J[J3_W0], w1 = J[J3_W1], w2 = J[J3_W2];
  const long long b0 = __float_as_int(J[J3_B0]);
  const long long b1 = SPH ? (long long)__float_as_int(J[J3_B1]) : 0;
  const long long s1 = SPH ? (long long)P.snr : (long long)P.n3x;
  const long long s2 = (long long)P.n3x * P.n3y;
#pragma unroll
  for (int c = 0; c < 8; c++) {
    const float w = ((c & 1) ? w0 : 1.0f - w0) * ((c & 2) ? w1 : 1.0f - w1) *
                    ((c & 4) ? w2 : 1.0f - w2);
    const long long id = SPH ? ((c & 4) ? b1 : b0) + (c & 1) + ((c >> 1) & 1) * s1
                             : b0 + (c & 1) + ((c >> 1) & 1) * s1 + (c >> 2) * s2;
    atomicAdd(G.g + id, make_float4(gT * w, gn * w, gv * w, gX * w));
    if (SPH) {
      const float lw = gl * w;
      atomicAdd(G.v + id, make_float4(lw * J[J3_ER], lw * J[J3_ETH], lw * J[J3_EPH], 0.0f));
    } else {
      atomicAdd(G.h + id, make_float2(gl * w, 0.0f));
    }
  }
}

// The 3-D grids' gradient copy (one copy) written out in FP64: {dT, dn, dvt, dX} per node and
// the velocity fields' gradients -- on the Cartesian grid from dL/dv_los (g2, the components'
// share of it is omega = (0, sin i, -cos i)), on the spherical grid as summed (v).
__global__ void grads3_kernel(const float4 *__restrict__ g4, const float2 *__restrict__ g2,
                              const float4 *__restrict__ v, long long n, double sin_i,
                              double cos_i, rt_grads3 G) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 a = g4[i];
    G.dT[i] = a.x;
    G.dn_h2[i] = a.y;
    G.dvturb[i] = a.z;
    G.dx_co[i] = a.w;
    if (v) {
      const float4 u = v[i];
      G.dvx[i] = u.x;
      G.dvy[i] = u.y;
      G.dvz[i] = u.z;
    } else {
      const double l = g2[i].x;
      G.dvx[i] = 0.0;
      G.dvy[i] = l * sin_i;
      G.dvz[i] = -l * cos_i;
    }
  }
}

// Channel window (as in the forward march): slot j of every lane is the channel block
// [LPR j, LPR j + LPR); bit j is set when some sample of the warp's batch has
// kd 2^{-d^2} >= 2^-40 in a channel of the block. Without equally spaced channels every block
// of a batch with gas is set. Skipped optical depths move a transmittance by less than 1e-9
// over a whole ray, and so do their terms of the gradients with respect to T, v_turb and the
// surfaces (all proportional to kd). The gradient with respect to the density is kd / n times
// these, which does not shrink with n where the density is tiny and the abundance is not (the
// top of the disk's wedge at large radii, the thin parts of a 3-D grid), so the window also
// keeps every channel where the profile is above 2^-20 of its peak (no measurable cost on the
// observation-scale disk: 1.145 -> 1.144 ms).
template <int LPR, int CPL>
__device__ __forceinline__ unsigned adj_window(const MarchParams &P, const float4 &mine,
                                               bool windowed, float idv) {
  if (!windowed) return __any_sync(0xffffffffu, mine.x > 0.0f) ? (1u << CPL) - 1 : 0u;
  float clo = 1.0f, chi = -1.0f;
  if (mine.x > 0.0f) {
    // never narrower than the channels where the profile is above 2^-20 of its peak, so that
    // a sample too thin for the absolute bound still has its gradient with respect to the
    // density (which does not shrink with it) computed to ~1e-6 of its own size
    const float w2 = fmaxf(40.0f + lg2(mine.x), 20.0f);
    if (w2 > 0.0f) {
      const float ib = rcp(mine.z);
      const float hw = sqa(w2) * ib;
      const float vl = mine.y * ib;  // v_los = a / b
      const float e0 = (vl - hw - P.v0) * idv, e1 = (vl + hw - P.v0) * idv;
      clo = fminf(e0, e1) - 0.01f;
      chi = fmaxf(e0, e1) + 0.01f;
    }
  }
  unsigned act = 0;
#pragma unroll
  for (int j = 0; j < CPL; j++)
    if (__any_sync(0xffffffffu, chi >= (float)(LPR * j) && clo <= (float)(LPR * j + LPR - 1)))
      act |= 1u << j;
  return act;
}

template <int LPR, int CPL, int VAR>
__global__ void __launch_bounds__(adj_wpb<LPR>() * 32, LPR >= 16 ? 7 : 4)
    march_adj_kernel(const __grid_constant__ MarchParams P, const float *__restrict__ dLdc,
                     const float *__restrict__ target, float *__restrict__ cube_out,
                     const rt_grads G, float *__restrict__ scratch, int nbat,
                     float4 *__restrict__ dmod, unsigned *__restrict__ dmax,
                     const GradCopies GC) {
  constexpr bool SPEC = (VAR & 4) != 0;  // the common configuration (spec_ok)
  constexpr bool UNIF = SPEC || (VAR & 1) != 0;  // equally spaced channels
  constexpr bool ROT = (VAR & 2) != 0;   // a rotation field (gradient with respect to it too)
  constexpr bool BOX = (VAR & 8) != 0;   // the 3-D Cartesian grid (rt_render3d_adjoint)
  constexpr bool SPH = (VAR & 16) != 0;  // the 3-D spherical grid (rt_render_sph_adjoint)
  constexpr bool GRID3 = BOX || SPH;
  constexpr bool VLOS = ROT || GRID3;    // dL/dv_los is needed (the sums az)
  constexpr bool CAP = GRID3;            // optical-depth increments capped at kDtCap
  constexpr int WPB = adj_wpb<LPR>();
  constexpr int R = 32 / LPR;          // rays per warp
  __shared__ __align__(16) float s_tab[kTabSeg * 4];
  // per ray LPR records plus one float4 of padding, so that the rays of a warp (reading one
  // record each, broadcast to their lanes) fall on different banks
  constexpr int kPhStride = LPR + 1;
  __shared__ float4 s_ph[WPB][(32 / LPR) * kPhStride];
  // per-sample channel sums of each lane, [sample t][lane ^ (t & 7)] (conflict-free both ways)
  __shared__ float4 s_part[WPB][LPR][32];
  // local derivatives of each lane's sample of the batch being reversed (physics_jac's
  // records, [slot][lane])
  __shared__ float4 s_rec[WPB][kRec][32];
  for (int i = threadIdx.x; i < kTabSeg * 4; i += blockDim.x) s_tab[i] = P.tab[i];
  __syncthreads();

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = lane % LPR, rr = lane / LPR;
  const long long npix = (long long)P.nx * P.ny;
  const long long nunits = (npix + R - 1) / R;
  const long long gw = (long long)blockIdx.x * WPB + wib;
  // this warp's scratch (adj_warp_floats): the depths at the end of the rays, the per-batch
  // entries and the batches' pair masks
  float *ck = scratch + gw * adj_warp_floats<LPR, CPL>(nbat);
  float2 *ent = reinterpret_cast<float2 *>(ck + CPL * 32) + lane;
  unsigned char *acts = reinterpret_cast<unsigned char *>(ck + CPL * 32 + (long long)nbat * (CPL / 2) * 64);
  float4 *rb = &s_rec[wib][0][lane];  // this lane's sample records
  float4 *ph = s_ph[wib];
  float4(*part)[32] = s_part[wib];
  float vc[CPL];
#pragma unroll
  for (int j = 0; j < CPL; j++)
    vc[j] = UNIF ? fmaf((float)(q + LPR * j), P.dv, P.v0) : P.v[min(q + LPR * j, RT_MAX_CH - 1)];
  const float vq = P.v0 + (float)q * P.dv;
  const float dvs = (float)LPR * P.dv;
  const bool windowed = UNIF && P.dv != 0.0f;
  const float idv = windowed ? 1.0f / P.dv : 0.0f;
  const float S_bg = P.I0 / P.out_scale;  // background in internal intensity units
  double loss = 0.0;
  float dmx = 0.0f;  // largest |dL/d(network output)| this lane wrote
  const GradSink Gb = block_sink(G, GC);
  // work counters (only with P.work): samples with gas, evaluations of the forward and reverse
  // passes
  unsigned long long wc_gas = 0, wc_fwd = 0, wc_rev = 0;

  // Dynamic work distribution: each warp takes the next unit (R neighbouring rays) from a
  // launch-wide counter, in pixel order, until none is left; the lanes set up their own ray
  // (about 1 % of a unit's work), so a warp that drew short rays simply takes more units and
  // the launch ends when the work does, not when the unluckiest warp's static share does.
  for (;;) {
    {
      unsigned uc = 0;
      if (lane == 0) uc = atomicAdd(P.unit_ctr, 1u);
      const long long u = (long long)__shfl_sync(0xffffffffu, uc, 0);
      if (u >= nunits) break;
      const long long pix = u * R + rr;
      const bool active = pix < npix;
      const Ray ray =
          setup_ray(P, active ? (int)(pix % P.nx) : 0, active ? (int)(pix / P.nx) : 0, active);
      // the rays' gas sample ranges (samples outside are exact no-ops), counted from klo;
      // batches and their kept depths are relative to it
      const int nsamp = __reduce_max_sync(0xffffffffu, max(ray.khi - ray.klo + 1, 0));

      // ---------- forward march, keeping the optical depth at every batch boundary ----------
      // channel slots in pairs (2m, 2m+1), packed two-lane FP32 instructions
      float2 tl[CPL / 2], tb[CPL / 2], Tr[CPL / 2], I[CPL / 2];
#pragma unroll
      for (int m = 0; m < CPL / 2; m++) {
        tl[m] = make_float2(0.0f, 0.0f);
        tb[m] = make_float2(0.0f, 0.0f);
        Tr[m] = make_float2(1.0f, 1.0f);
        I[m] = make_float2(0.0f, 0.0f);
      }
      const float2 mone = make_float2(-1.0f, -1.0f);
      int nent = 0;  // entries kept (warp-uniform)
      for (int kb = 0; kb < nsamp; kb += LPR) {
        float4 mine;
        if constexpr (SPH)
          mine = sample_physics_sph(P, s_tab, ray, ray.klo + kb + q);
        else if constexpr (BOX)
          mine = sample_physics_box(P, s_tab, ray, ray.klo + kb + q);
        else
          mine = sample_physics<ROT, SPEC>(P, s_tab, ray, ray.klo + kb + q);
        const unsigned act = adj_window<LPR, CPL>(P, mine, windowed, idv);
        unsigned act2 = 0;
#pragma unroll
        for (int m = 0; m < CPL / 2; m++)
          if ((act >> (2 * m)) & 3u) act2 |= 1u << m;
        if (lane == 0) acts[kb / LPR] = (unsigned char)act2;  // (the reverse marches these)
        if (P.work) {
          wc_gas += __popc(__ballot_sync(0xffffffffu, mine.x > 0.0f));
          wc_fwd += (unsigned long long)__popc(act2) * 2 * LPR * 32;
        }
        if (!act) continue;
        ph[rr * kPhStride + q] = mine;
        __syncwarp();
        // channel pairs outside, the batch's samples inside: one warp-uniform window test per
        // pair and batch
#pragma unroll
        for (int m = 0; m < CPL / 2; m++) {
          if (!(act2 & (1u << m))) continue;  // warp-uniform
#pragma unroll
          for (int t = 0; t < LPR; t++) {
            const float4 p = ph[rr * kPhStride + t];
            const float dc = fmaf(vq, p.z, -p.y), db = __fmul_rn(dvs, p.z);
            const float2 kd2 = make_float2(p.x, p.x), S2 = make_float2(p.w, p.w);
            const float2 d =
                UNIF ? __ffma2_rn(make_float2((float)(2 * m), (float)(2 * m + 1)),
                                  make_float2(db, db), make_float2(dc, dc))
                     : __ffma2_rn(make_float2(vc[2 * m], vc[2 * m + 1]),
                                  make_float2(p.z, p.z), make_float2(-p.y, -p.y));
            const float2 d2 = __fmul2_rn(d, d);
            if constexpr (CAP) {
              const float2 dt = __fmul2_rn(kd2, make_float2(ex2(-d2.x), ex2(-d2.y)));
              tl[m] = __fadd2_rn(tl[m], make_float2(fminf(dt.x, kDtCap), fminf(dt.y, kDtCap)));
            } else {
              tl[m] = __ffma2_rn(kd2, make_float2(ex2(-d2.x), ex2(-d2.y)), tl[m]);
            }
            const float2 nt = __fadd2_rn(tb[m], tl[m]);
            const float2 Tn = make_float2(ex2(-nt.x), ex2(-nt.y));
            I[m] = __ffma2_rn(S2, __ffma2_rn(Tn, mone, Tr[m]), I[m]);
            Tr[m] = Tn;
          }
        }
        // compensated fold of the batch into the base of the pairs it advanced (Kahan, as in
        // the forward march; the other pairs' sums did not change): tl carries the batch sum
        // minus the rounding error of the previous fold. Their depths at the batch end (the
        // base plus the compensation the fold left in tl) are kept: one entry per pair, in
        // pair order.
#pragma unroll
        for (int m = 0; m < CPL / 2; m++)
          if (act2 & (1u << m)) {  // warp-uniform
            const float2 t = __fadd2_rn(tb[m], tl[m]);
            tl[m] = __ffma2_rn(__ffma2_rn(tb[m], mone, t), mone, tl[m]);
            tb[m] = t;
            ent[(long long)nent * 32] = make_float2(tb[m].x + tl[m].x, tb[m].y + tl[m].y);
            nent++;
          }
        __syncwarp();
      }
      {  // the depths at the end of the rays
        float4 *o = reinterpret_cast<float4 *>(ck + lane * CPL);
#pragma unroll
        for (int m = 0; m < CPL / 2; m += 2)
          o[m / 2] = make_float4(tb[m].x + tl[m].x, tb[m].y + tl[m].y, tb[m + 1].x + tl[m + 1].x,
                                 tb[m + 1].y + tl[m + 1].y);
      }
      __syncwarp();  // (lane 0's pair masks, for every lane's reverse pass)

      // ---------------- loss seed ----------------
      float2 gI[CPL / 2];  // dL/d(internal intensity) of slots (2m, 2m+1)
#pragma unroll
      for (int j = 0; j < CPL; j++) {
        const int ch = q + LPR * j;
        float go = 0.0f;
        if (active && ch < P.nch) {
          const long long o = (long long)ch * npix + pix;
          const float Ij = (j & 1) ? I[j >> 1].y : I[j >> 1].x;
          const float Trj = (j & 1) ? Tr[j >> 1].y : Tr[j >> 1].x;
          const float out = fmaf(Ij, P.out_scale, P.I0 * Trj);
          if (cube_out) __stcs(cube_out + o, out);
          // read once: streamed past L2 (evict first), which keeps the per-warp scratch and
          // the gradient copies resident
          if (dLdc) {
            go = __ldcs(dLdc + o);
          } else {
            const float r = out - __ldcs(target + o);
            go = 2.0f * r;
            loss += (double)r * (double)r;
          }
        }
        if (j & 1)
          gI[j >> 1].y = go * P.out_scale;
        else
          gI[j >> 1].x = go * P.out_scale;
      }
      if (nsamp == 0) continue;

      // ---------------- reverse march, batch by batch (last to first) ----------------
      float2 A[CPL / 2];  // suffix sums of channel slots (2m, 2m+1)
#pragma unroll
      for (int m = 0; m < CPL / 2; m++) A[m] = make_float2(0.0f, 0.0f);
      float Snext = S_bg;
      // optical depths and transmittances of the channel pairs at the end of the batch being
      // reversed: the forward pass's values for the pairs the batch advances; the other pairs
      // carry theirs from the later batches (unchanged in between)
      float2 cur[CPL / 2], Tn[CPL / 2];
      {
        const float4 *ce = reinterpret_cast<const float4 *>(ck + lane * CPL);
#pragma unroll
        for (int m = 0; m < CPL / 2; m += 2) {
          const float4 v = ce[m / 2];
          cur[m] = make_float2(v.x, v.y);
          cur[m + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int m = 0; m < CPL / 2; m++) Tn[m] = make_float2(ex2(-cur[m].x), ex2(-cur[m].y));
      }
      int ient = nent;
      const int blast = (nsamp + LPR - 1) / LPR - 1;
      unsigned act_next = blast >= 0 ? acts[blast] : 0u;  // read a batch ahead
      for (int b = blast; b >= 0; b--) {
        const int kb = b * LPR;
        // the channel pairs the forward pass advanced in this batch (the same window), whose
        // entries precede the later batches'
        const unsigned act2 = act_next;
        if (b > 0) act_next = acts[b - 1];
        ient -= __popc(act2);
        // the kept depths of those pairs, loaded before the sample's physics so that their L2
        // latency overlaps it (a batch without gas advanced no pair and loads nothing)
        {
          int e = ient;
#pragma unroll
          for (int m = 0; m < CPL / 2; m++)
            if (act2 & (1u << m)) {  // warp-uniform
              cur[m] = ent[(long long)e * 32];
              e++;
            }
        }
        // physics and local derivatives of this lane's sample (records in shared memory, read
        // back by the same lane for its chain rule)
        float4 mine;
        if constexpr (SPH)
          mine = physics_jac_sph(P, s_tab, ray, ray.klo + kb + q, rb);
        else if constexpr (BOX)
          mine = physics_jac_box(P, s_tab, ray, ray.klo + kb + q, rb);
        else
          mine = physics_jac<ROT, SPEC>(P, s_tab, ray, ray.klo + kb + q, rb);
        if (!__any_sync(0xffffffffu, mine.z > 0.0f)) continue;  // no gas in the batch
        const float Sbefore = Snext;
        ph[rr * kPhStride + q] = mine;
        if (P.work) wc_rev += (unsigned long long)__popc(act2) * 2 * LPR * 32;
#pragma unroll
        for (int m = 0; m < CPL / 2; m++)
          if (act2 & (1u << m)) Tn[m] = make_float2(ex2(-cur[m].x), ex2(-cur[m].y));
        __syncwarp();
        const float2 mone = make_float2(-1.0f, -1.0f);
        // reverse step of one channel pair m at sample t of the batch: advances the suffix
        // sums A, the optical depth cur and the transmittance Tn of the pair, and returns its
        // contributions to the per-sample channel sums (ax, ay, az, aw)
        auto rev_step = [&](int m, const float4 &p, float cs) {
          const float dc = fmaf(vq, p.z, -p.y), db = __fmul_rn(dvs, p.z);
          const float2 cs2 = make_float2(cs, cs), kd2 = make_float2(p.x, p.x);
          const float2 d =
              UNIF ? __ffma2_rn(make_float2((float)(2 * m), (float)(2 * m + 1)),
                                make_float2(db, db), make_float2(dc, dc))
                   : __ffma2_rn(make_float2(vc[2 * m], vc[2 * m + 1]),
                                make_float2(p.z, p.z), make_float2(-p.y, -p.y));
          const float2 d2 = __fmul2_rn(d, d);
          const float2 gg = make_float2(ex2(-d2.x), ex2(-d2.y));
          A[m] = __ffma2_rn(cs2, Tn[m], A[m]);
          const float2 ug = __fmul2_rn(__fmul2_rn(gI[m], A[m]), gg);
          float2 dt = __fmul2_rn(kd2, gg);
          if constexpr (CAP) dt = make_float2(fminf(dt.x, kDtCap), fminf(dt.y, kDtCap));
          cur[m] = __ffma2_rn(dt, mone, cur[m]);
          const float2 T0 = make_float2(ex2(-cur[m].x), ex2(-cur[m].y));
          // T_k - T_{k+1} = T_{k+1} (2^dt - 1): series below dt = 0.07 (the difference of
          // two rounded transmittances would lose the small optical depths)
          const float2 poly = __ffma2_rn(
              __ffma2_rn(dt, make_float2(0.0555041087f, 0.0555041087f),
                         make_float2(0.240226507f, 0.240226507f)),
              dt, make_float2(0.693147181f, 0.693147181f));
          const float2 ser = __fmul2_rn(__fmul2_rn(Tn[m], dt), poly);
          const float2 dif = __ffma2_rn(Tn[m], mone, T0);
          const float2 dTk = make_float2(dt.x < 0.07f ? ser.x : dif.x,
                                         dt.y < 0.07f ? ser.y : dif.y);
          Tn[m] = T0;
          const float2 wy = __fmul2_rn(ug, d2), wz = __fmul2_rn(ug, d), ww = __fmul2_rn(gI[m], dTk);
          return make_float4(ug.x + ug.y, wy.x + wy.y, VLOS ? wz.x + wz.y : 0.0f, ww.x + ww.y);
        };
        // one channel pair in the window (the common case): its loop without per-sample
        // window tests, the pair index a compile-time constant
        auto one_pair = [&](auto M) {
          constexpr int m = decltype(M)::value;
#pragma unroll 1
          for (int t = LPR - 1; t >= 0; t--) {
            const float4 p = ph[rr * kPhStride + t];
            const bool gas = p.z > 0.0f;
            const float cs = gas ? Snext - p.w : 0.0f;  // S_{k+1} - S_k
            Snext = gas ? p.w : Snext;
            part[t][lane ^ (t & 7)] = rev_step(m, p, cs);
          }
        };
        // two adjacent pairs in the window (the next most common case), likewise
        auto two_pairs = [&](auto M) {
          constexpr int m = decltype(M)::value;
#pragma unroll 1
          for (int t = LPR - 1; t >= 0; t--) {
            const float4 p = ph[rr * kPhStride + t];
            const bool gas = p.z > 0.0f;
            const float cs = gas ? Snext - p.w : 0.0f;  // S_{k+1} - S_k
            Snext = gas ? p.w : Snext;
            const float4 c0 = rev_step(m, p, cs), c1 = rev_step(m + 1, p, cs);
            part[t][lane ^ (t & 7)] =
                make_float4(c0.x + c1.x, c0.y + c1.y, c0.z + c1.z, c0.w + c1.w);
          }
        };
        const int npair = __popc(act2);
        if (npair == 2 && act2 == 3u) {
          two_pairs(std::integral_constant<int, 0>());
        } else if (CPL / 2 > 2 && npair == 2 && act2 == 6u) {
          two_pairs(std::integral_constant<int, (CPL / 2 > 2 ? 1 : 0)>());
        } else if (CPL / 2 > 3 && npair == 2 && act2 == 12u) {
          two_pairs(std::integral_constant<int, (CPL / 2 > 3 ? 2 : 0)>());
        } else if (npair == 1 && act2 == 1u) {
          one_pair(std::integral_constant<int, 0>());
        } else if (npair == 1 && act2 == 2u) {
          one_pair(std::integral_constant<int, 1>());
        } else if (CPL / 2 > 2 && npair == 1 && act2 == 4u) {
          one_pair(std::integral_constant<int, (CPL / 2 > 2 ? 2 : 0)>());
        } else if (CPL / 2 > 3 && npair == 1 && act2 == 8u) {
          one_pair(std::integral_constant<int, (CPL / 2 > 3 ? 3 : 0)>());
        } else {
#pragma unroll 1
          for (int t = LPR - 1; t >= 0; t--) {
            const float4 p = ph[rr * kPhStride + t];
            const bool gas = p.z > 0.0f;
            const float cs = gas ? Snext - p.w : 0.0f;  // S_{k+1} - S_k
            Snext = gas ? p.w : Snext;
            float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int m = 0; m < CPL / 2; m++) {
              if (!(act2 & (1u << m))) continue;  // warp-uniform
              const float4 c = rev_step(m, p, cs);
              a.x += c.x;
              a.y += c.y;
              a.z += c.z;
              a.w += c.w;
            }
            part[t][lane ^ (t & 7)] = a;
          }
        }
        // blocks outside every window: T is constant over the batch, so the suffix sums
        // advance by T (S before the batch - S of its first sample with gas)
        const float dS = Sbefore - Snext;
#pragma unroll
        for (int m = 0; m < CPL / 2; m++)
          if (!(act2 & (1u << m))) A[m] = __ffma2_rn(make_float2(dS, dS), Tn[m], A[m]);
        __syncwarp();
        float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 8
        for (int i = 0; i < LPR; i++) {
          const float4 v = part[q][(rr * LPR + i) ^ (q & 7)];
          s.x += v.x;
          s.y += v.y;
          if (VLOS) s.z += v.z;
          s.w += v.w;
        }
        if (active && mine.z > 0.0f) {
          float Jv[4 * (kRec - 1)];
#pragma unroll
          for (int i = 0; i < kRec - 1; i++) {
            const float4 v = (i < kRec - 2 || (!SPEC && P.mod) || ROT || SPH) ? rb[(i + 1) * 32]
                                                            : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
            Jv[4 * i] = v.x;
            Jv[4 * i + 1] = v.y;
            Jv[4 * i + 2] = v.z;
            Jv[4 * i + 3] = v.w;
          }
          if constexpr (GRID3)
            scatter_3d<SPH>(P, Jv, mine.x, mine.z, s.x, s.y, s.z, s.w, Gb);
          else
            dmx = fmaxf(dmx, scatter_grad<ROT>(P, Jv, mine.x, mine.z, s.x, s.y, s.z, s.w, Gb,
                                          dmod ? dmod + (long long)pix * P.n_samples + ray.klo + kb + q
                                               : nullptr));
        }
        __syncwarp();
      }
    }
  }
  if (P.work && lane == 0) {
    atomicAdd(P.work, wc_gas);
    atomicAdd(P.work + 1, wc_fwd);
    atomicAdd(P.work + 3, wc_rev);
  }
  if (G.loss && target) {
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if (lane == 0 && loss != 0.0) atomicAdd(G.loss, loss);
  }
  if (dmax) {
    for (int o = 16; o > 0; o >>= 1) dmx = fmaxf(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
    if (lane == 0 && dmx > 0.0f) atomicMax(dmax, __float_as_uint(dmx));
  }
}

// Kernel variant of a problem: bit 0 equally spaced channels, bit 1 a rotation field; the
// common configuration without a rotation field (spec_ok, checked after the corner quads are
// planned) takes variant 5, specialised for it.
static int adj_variant(const MarchParams &P) {
  return (P.v_uniform ? 1 : 0) | (P.vphi ? 2 : 0);
}

// Lane layout of the adjoint: CPL channels per lane (8 from 32 channels up), LPR lanes per
// ray (a power of two, at least 2).
void adj_layout(int nch, int *lpr, int *cpl) {
  int c = nch >= 32 ? 8 : 4;
  int need = (nch + c - 1) / c;
  int l = 2;
  while (l < need) l <<= 1;
  *lpr = l;
  *cpl = c;
}

// Chain rule to power-law surface parameters (one block).
__global__ void surface_powerlaw_kernel(int nr, int r_log, double r_in, double r_out,
                                        const double *__restrict__ dh,
                                        const float *__restrict__ h, double c,
                                        double *__restrict__ out) {
  __shared__ double s_c[256], s_p[256];
  double ac = 0.0, ap = 0.0;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    double t = (double)i / (nr - 1);
    double r = r_log ? r_in * pow(r_out / r_in, t) : r_in + (r_out - r_in) * t;
    double gh = dh[i] * (double)h[i];
    ac += gh / c;
    ap += gh * log(r / 100.0);
  }
  s_c[threadIdx.x] = ac;
  s_p[threadIdx.x] = ap;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_c[threadIdx.x] += s_c[threadIdx.x + s];
      s_p[threadIdx.x] += s_p[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_c[0];
    out[1] = s_p[0];
  }
}

// Layouts the adjoint is compiled for (lanes per ray, channels per lane); adj_layout picks one.
#define RTB_ADJ_LAYOUTS(X) X(2, 4) X(4, 4) X(8, 4) X(4, 8) X(8, 8) X(16, 8) X(32, 8)

// Blocks of the persistent grid of the adjoint kernel for P (cap_blocks <= 0 asks the
// occupancy calculator).
template <int LPR, int CPL, int VAR>
static long long adj_blocks(const MarchParams &P, long long cap_blocks) {
  constexpr int WPB = adj_wpb<LPR>();
  long long npix = (long long)P.nx * P.ny;
  long long units = (npix + (32 / LPR) - 1) / (32 / LPR);
  long long need = (units + WPB - 1) / WPB;
  long long cap = cap_blocks > 0
                      ? cap_blocks
                      : resident_blocks((const void *)march_adj_kernel<LPR, CPL, VAR>, WPB * 32);
  return need < cap ? need : cap;
}

// Bytes of per-warp scratch (the depths kept at the batch boundaries and the batches' pair
// masks; "checkpoints" below) one block needs.
template <int LPR, int CPL>
static size_t adj_block_bytes(const MarchParams &P) {
  return (size_t)adj_wpb<LPR>() * adj_warp_floats<LPR, CPL>(adj_batches<LPR>(P.n_samples)) *
         sizeof(float);
}

// Scratch of one adjoint launch: the warps' checkpoints, the gradient copies, then the
// corner quads of the fields (cell_bytes; 0 when the kernel reads the node arrays).
struct AdjScratch {
  size_t ck_bytes, g_off, h_off, cell_off, cell_bytes, ctr_off, total;
  int kg, kh;
};

constexpr size_t kCopyBudget = (size_t)16 << 20;  // bytes of grid-gradient copies at most
constexpr int kMaxGridCopies = 32;
constexpr int kMaxSurfCopies = 128;

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout for `blocks` blocks with ck_bytes of checkpoints; gradient copies within `avail`
// bytes in total (0: no limit).
static AdjScratch plan_scratch(const MarchParams &P, long long blocks, size_t ck_bytes,
                               size_t avail) {
  AdjScratch a;
  a.ck_bytes = align256(ck_bytes);
  const size_t gcopy = (size_t)P.nr * P.nz * sizeof(float4);
  const size_t hcopy = (size_t)P.nr * sizeof(float2);
  long long kg = (long long)(kCopyBudget / gcopy);
  if (kg > kMaxGridCopies) kg = kMaxGridCopies;
  if (kg > blocks) kg = blocks;
  long long kh = kMaxSurfCopies < blocks ? kMaxSurfCopies : blocks;
  a.cell_bytes = align256(cell_bytes(P));
  if (avail) {
    // surface copies first (small, and without them every radius serializes), then the
    // corner quads, then grid copies in what is left
    size_t left = avail > a.ck_bytes + 256 ? avail - a.ck_bytes - 256 : 0;  // (the counter)
    while (kh > 0 && (size_t)kh * hcopy > left / 4) kh /= 2;
    left -= align256((size_t)kh * hcopy);
    if (a.cell_bytes + 256 > left) a.cell_bytes = 0;
    left -= a.cell_bytes;
    while (kg > 0 && (size_t)kg * gcopy + 256 > left) kg /= 2;
  }
  a.kg = kg > 1 ? (int)kg : 0;  // one copy buys nothing over the caller's arrays
  a.kh = kh > 1 ? (int)kh : 0;
  a.g_off = a.ck_bytes;
  a.h_off = a.g_off + align256((size_t)a.kg * gcopy);
  a.cell_off = a.h_off + align256((size_t)a.kh * hcopy);
  a.ctr_off = a.cell_off + a.cell_bytes;  // the work counter of the dynamic distribution
  a.total = a.ctr_off + 256;
  return a;
}

static int zero_grads(const MarchParams &P, const rt_grads &G, const AdjScratch &a,
                      char *scratch, cudaStream_t stream) {
  size_t ng = (size_t)P.nr * P.nz * sizeof(double), nh = (size_t)P.nr * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (a.kg) {
    e = cudaMemsetAsync(scratch + a.g_off, 0, a.h_off - a.g_off, stream);
  } else {
    e = cudaMemsetAsync(G.dT, 0, ng, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(G.dn, 0, ng, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(G.dvt, 0, ng, stream);
    if (e == cudaSuccess && P.vphi) e = cudaMemsetAsync(G.dvphi, 0, ng, stream);
  }
  if (e == cudaSuccess && a.kh) {
    e = cudaMemsetAsync(scratch + a.h_off, 0, a.cell_off - a.h_off, stream);
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(G.dh_lo, 0, nh, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(G.dh_hi, 0, nh, stream);
  }
  if (e == cudaSuccess && G.loss) e = cudaMemsetAsync(G.loss, 0, sizeof(double), stream);
  if (e == cudaSuccess && scratch) e = cudaMemsetAsync(scratch + a.ctr_off, 0, 256, stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "gradient memset: %s", cudaGetErrorString(e));
  return RT_OK;
}

static GradCopies copies_of(const MarchParams &P, const AdjScratch &a, char *scratch) {
  GradCopies c;
  c.g = a.kg ? reinterpret_cast<float4 *>(scratch + a.g_off) : nullptr;
  c.h = a.kh ? reinterpret_cast<float2 *>(scratch + a.h_off) : nullptr;
  c.gstride = (long long)P.nr * P.nz;
  c.hstride = P.nr;
  c.kg = a.kg > 0 ? a.kg : 1;
  c.kh = a.kh > 0 ? a.kh : 1;
  c.v = nullptr;
  return c;
}

static int sum_copies(const MarchParams &P, const rt_grads &G, const GradCopies &c,
                      const AdjScratch &a, cudaStream_t stream) {
  if (a.kg) {
    long long m = (long long)P.nr * P.nz;
    long long nb = (m + 255) / 256;
    sum_grid_copies_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, stream>>>(
        c.g, a.kg, c.gstride, m, G.dT, G.dn, G.dvt, P.vphi ? G.dvphi : nullptr);
  }
  if (a.kh) {
    long long nb = (P.nr + 7) / 8;  // 8 warps (entries) per block
    sum_surface_copies_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, stream>>>(
        c.h, a.kh, c.hstride, P.nr, G.dh_lo, G.dh_hi);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "gradient sum: %s", cudaGetErrorString(e));
  return RT_OK;
}

// Zero, march, sum: one adjoint launch on `scratch` (laid out by a).
template <int LPR, int CPL, int VAR>
static int run_adj(const MarchParams &P, const float *dLdc, const float *target, float *cube_out,
                   const rt_grads &G, float4 *dmod, unsigned *dmax, long long blocks,
                   const AdjScratch &a, char *scratch, cudaStream_t stream) {
  int rc = zero_grads(P, G, a, scratch, stream);
  if (rc != RT_OK) return rc;
  const GradCopies c = copies_of(P, a, scratch);
  const int nbat = adj_batches<LPR>(P.n_samples);
  // the kernel takes the parameters by value, so the copy pointing at the corner quads only
  // has to live until the launch (on the stack: no host allocation)
  MarchParams Q = P;
  Q.rays = nullptr;
  Q.unit_ctr = reinterpret_cast<unsigned *>(scratch + a.ctr_off);
  if (a.cell_bytes) {
    rc = pack_cells(Q, scratch + a.cell_off, stream);
    if (rc != RT_OK) return rc;
  }
  bool launched = false;
  if constexpr (VAR == 1) {
    if (spec_ok(Q)) {  // the specialised variant (same scratch layout and block count)
      march_adj_kernel<LPR, CPL, 5><<<(unsigned)blocks, adj_wpb<LPR>() * 32, 0, stream>>>(
          Q, dLdc, target, cube_out, G, reinterpret_cast<float *>(scratch), nbat, dmod, dmax, c);
      launched = true;
    }
  }
  if (!launched)
    march_adj_kernel<LPR, CPL, VAR><<<(unsigned)blocks, adj_wpb<LPR>() * 32, 0, stream>>>(
        Q, dLdc, target, cube_out, G, reinterpret_cast<float *>(scratch), nbat, dmod, dmax, c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "adjoint launch: %s", cudaGetErrorString(e));
  return sum_copies(P, G, c, a, stream);
}

template <int LPR, int CPL, int VAR>
static int launch_adj_t(const MarchParams &P, const float *dLdc, const float *target,
                        float *cube_out, const rt_grads &G, float4 *dmod, unsigned *dmax,
                        cudaStream_t stream) {
  const long long blocks = adj_blocks<LPR, CPL, VAR>(P, 0);
  const AdjScratch a = plan_scratch(P, blocks, blocks * adj_block_bytes<LPR, CPL>(P), 0);
  char *scratch = nullptr;
  cudaError_t e = stream_alloc((void **)&scratch, a.total, stream);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "adjoint scratch (%zu bytes): %s", a.total,
                     cudaGetErrorString(e));
  int rc = run_adj<LPR, CPL, VAR>(P, dLdc, target, cube_out, G, dmod, dmax, blocks, a,
                                   scratch, stream);
  cudaFreeAsync(scratch, stream);
  return rc;
}

// Launches the fused adjoint (the gradient outputs are overwritten, not accumulated into).
// dmod (optional, [pixel][sample] float4) receives dL/d(network outputs) for samples with gas
// and is left untouched elsewhere; dmax (optional, zeroed by the caller) their largest
// magnitude as float bits.
int launch_adjoint(const MarchParams &P, const float *dLdc, const float *target,
                   float *cube_out, const rt_grads &G, cudaStream_t stream, float4 *dmod,
                   unsigned *dmax) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return zero_grads(P, G, plan_scratch(P, 1, 0, 0), nullptr, stream);
  int LPR, CPL;
  adj_layout(P.nch, &LPR, &CPL);
  const int v = adj_variant(P);
#define X(L, C)                                                                         \
  if (LPR == L && CPL == C) {                                                           \
    if (v == 0) return launch_adj_t<L, C, 0>(P, dLdc, target, cube_out, G, dmod, dmax, stream); \
    if (v == 1) return launch_adj_t<L, C, 1>(P, dLdc, target, cube_out, G, dmod, dmax, stream); \
    if (v == 2) return launch_adj_t<L, C, 2>(P, dLdc, target, cube_out, G, dmod, dmax, stream); \
    return launch_adj_t<L, C, 3>(P, dLdc, target, cube_out, G, dmod, dmax, stream);     \
  }
  RTB_ADJ_LAYOUTS(X)
#undef X
  return set_error(RT_EINVAL, "no adjoint layout for %d channels", P.nch);
}

// The adjoint on a 3-D grid (P.box or P.sph, node records in P.node_a / node_b): scratch for
// the kept optical depths, one FP32 gradient copy ({dT, dn, dvt, dX} per node, and {dv_los, 0}
// per node on the Cartesian grid or {dv_r, dv_theta, dv_phi, 0} on the spherical one) and the
// work counter; zero, march, write the FP64 gradients.
template <int LPR, int CPL, int VAR>
static int launch_adj3_t(const MarchParams &P, const float *dLdc, const float *target,
                         float *cube_out, const rt_grads3 &G3, cudaStream_t stream) {
  constexpr bool SPH = (VAR & 16) != 0;
  const long long nodes = SPH ? (long long)P.snr * P.snth * P.snph
                              : (long long)P.n3x * P.n3y * P.n3z;
  const long long blocks = adj_blocks<LPR, CPL, VAR>(P, 0);
  const size_t ck = align256((size_t)blocks * adj_block_bytes<LPR, CPL>(P));
  const size_t g4 = align256((size_t)nodes * sizeof(float4));
  const size_t g2 = align256((size_t)nodes * (SPH ? sizeof(float4) : sizeof(float2)));
  char *scratch = nullptr;
  cudaError_t e = stream_alloc((void **)&scratch, ck + g4 + g2 + 256, stream);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "adjoint scratch (%zu bytes): %s", ck + g4 + g2 + 256,
                     cudaGetErrorString(e));
  e = cudaMemsetAsync(scratch + ck, 0, g4 + g2 + 256, stream);  // copy and counter
  if (e == cudaSuccess && G3.loss) e = cudaMemsetAsync(G3.loss, 0, sizeof(double), stream);
  int rc = RT_OK;
  if (e != cudaSuccess) rc = set_error(RT_ECUDA, "gradient memset: %s", cudaGetErrorString(e));
  if (rc == RT_OK) {
    GradCopies c;
    c.g = reinterpret_cast<float4 *>(scratch + ck);
    c.h = SPH ? nullptr : reinterpret_cast<float2 *>(scratch + ck + g4);
    c.v = SPH ? reinterpret_cast<float4 *>(scratch + ck + g4) : nullptr;
    c.gstride = c.hstride = nodes;
    c.kg = c.kh = 1;
    rt_grads G = {};
    G.loss = G3.loss;
    MarchParams Q = P;
    Q.rays = nullptr;
    Q.unit_ctr = reinterpret_cast<unsigned *>(scratch + ck + g4 + g2);
    march_adj_kernel<LPR, CPL, VAR><<<(unsigned)blocks, adj_wpb<LPR>() * 32, 0, stream>>>(
        Q, dLdc, target, cube_out, G, reinterpret_cast<float *>(scratch),
        adj_batches<LPR>(P.n_samples), nullptr, nullptr, c);
    const long long nb = (nodes + 255) / 256;
    grads3_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, stream>>>(
        c.g, c.h, c.v, nodes, (double)P.sin_if, (double)P.cos_if, G3);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = set_error(RT_ECUDA, "3-D adjoint launch: %s", cudaGetErrorString(e));
  }
  cudaFreeAsync(scratch, stream);
  return rc;
}

int launch_adjoint3(const MarchParams &P, const float *dLdc, const float *target,
                    float *cube_out, const rt_grads3 &G3, cudaStream_t stream) {
  int LPR, CPL;
  adj_layout(P.nch, &LPR, &CPL);
#define X(L, C)                                                                            \
  if (LPR == L && CPL == C) {                                                              \
    if (P.sph)                                                                             \
      return P.v_uniform ? launch_adj3_t<L, C, 17>(P, dLdc, target, cube_out, G3, stream)  \
                         : launch_adj3_t<L, C, 16>(P, dLdc, target, cube_out, G3, stream); \
    return P.v_uniform ? launch_adj3_t<L, C, 9>(P, dLdc, target, cube_out, G3, stream)     \
                       : launch_adj3_t<L, C, 8>(P, dLdc, target, cube_out, G3, stream);    \
  }
  RTB_ADJ_LAYOUTS(X)
#undef X
  return set_error(RT_EINVAL, "no adjoint layout for %d channels", P.nch);
}

// Scratch rt_render_adjoint allocates for P (cap_blocks > 0 replaces the device occupancy
// query, for planning without a GPU).
size_t adjoint_scratch_bytes(const MarchParams &P, long long cap_blocks) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return 0;
  int LPR, CPL;
  adj_layout(P.nch, &LPR, &CPL);
  long long b = 1;
  size_t per = 0;
  const int v = adj_variant(P);
#define X(L, C)                                                                            \
  if (LPR == L && CPL == C) {                                                              \
    b = v == 0 ? adj_blocks<L, C, 0>(P, cap_blocks)                                        \
               : v == 1 ? adj_blocks<L, C, 1>(P, cap_blocks)                               \
                        : v == 2 ? adj_blocks<L, C, 2>(P, cap_blocks)                      \
                                 : adj_blocks<L, C, 3>(P, cap_blocks);                     \
    per = adj_block_bytes<L, C>(P);                                                        \
  }
  RTB_ADJ_LAYOUTS(X)
#undef X
  return plan_scratch(P, b, b * per, 0).total;
}

int launch_surface_grad(const rt_grid &g, const double *dh, const float *h, double c,
                        double *out, cudaStream_t stream) {
  surface_powerlaw_kernel<<<1, 256, 0, stream>>>(g.nr, g.r_log, g.r_in_au, g.r_out_au, dh, h,
                                                 c, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "surface gradient: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rtb

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the adjoint entry point.
//
// Some callers cannot call cudaMalloc (or have it called on their behalf): for example an
// application whose own memory manager has already reserved the device's memory, or a
// service that runs under a fixed device-memory budget and forbids allocator traffic once it
// is running. For them the scratch of the adjoint (checkpoints, then as many gradient copies
// and, room permitting, the corner quads of the fields) lives in one file-scope device array of fixed size, kFixedScratchBytes, that every
// GPU loading this library holds until the process exits. The kernel is the same; when the
// array cannot hold a checkpoint region for every resident block, the persistent grid is
// made smaller, and where fewer gradient copies fit (or none: then the blocks add straight
// into the caller's arrays) the FP64 sums run in another order: same results, lower
// throughput. A problem whose single block does not fit is rejected.
// ---------------------------------------------------------------------------------------
namespace rtb {

constexpr size_t kFixedScratchBytes = (size_t)32 << 20;  // 32 MiB per device
static __device__ __align__(256) float g_fixed_scratch[kFixedScratchBytes / sizeof(float)];

// Unique ID of the CUDA context current on this thread (0 where none is current or the query
// is unavailable), through the driver entry points the runtime hands out (no link-time
// dependency on the driver library).
static unsigned long long current_context_id() {
  typedef int (*GetCurrent)(void **);
  typedef int (*GetId)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult st;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &st) ==
            cudaSuccess &&
        st == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &st) ==
            cudaSuccess &&
        st == cudaDriverEntryPointSuccess) {
      get_current = (GetCurrent)f;
      get_id = (GetId)g;
    }
  });
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_fixed_scratch in the current device's context. The host-side name is
// only a stand-in for the symbol, so the address is looked up with that device current and
// cached per device together with the ID of the context it belongs to; a different context
// (after cudaDeviceReset, say, the library's module is loaded anew) triggers a new lookup.
static int fixed_scratch_address(float **out) {
  struct Entry {
    unsigned long long ctx;
    float *addr;
  };
  static std::mutex mu;
  static Entry cache[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(RT_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(mu);
  const unsigned long long ctx = current_context_id();
  if (!cache[dev].addr || ctx == 0 || cache[dev].ctx != ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fixed_scratch);  // also initialises the context if needed
    if (e != cudaSuccess || !p)
      return set_error(RT_ECUDA, "cudaGetSymbolAddress(fixed scratch): %s", cudaGetErrorString(e));
    cache[dev].addr = (float *)p;
    cache[dev].ctx = ctx ? ctx : current_context_id();
  }
  *out = cache[dev].addr;
  return RT_OK;
}

template <int LPR, int CPL, int VAR>
static int launch_adj_fixed_t(const MarchParams &P, const float *dLdc, const float *target,
                              float *cube_out, const rt_grads &G, cudaStream_t stream,
                              float *scratch) {
  // checkpoints get at most three quarters of the array; surface copies, corner quads and
  // grid copies share what is left
  const size_t ck_room = kFixedScratchBytes / 4 * 3;
  const size_t per_block = adj_block_bytes<LPR, CPL>(P);
  if (per_block > ck_room)
    return set_error(RT_EINVAL,
                     "allocation-free adjoint: %d samples per ray need %zu bytes of checkpoint "
                     "scratch per block, above the %zu bytes the fixed array gives them",
                     P.n_samples, per_block, ck_room);
  long long blocks = adj_blocks<LPR, CPL, VAR>(P, 0);
  const long long fit = (long long)(ck_room / per_block);
  if (blocks > fit) blocks = fit;
  const AdjScratch a = plan_scratch(P, blocks, blocks * per_block, kFixedScratchBytes);
  return run_adj<LPR, CPL, VAR>(P, dLdc, target, cube_out, G, nullptr, nullptr, blocks, a,
                                 reinterpret_cast<char *>(scratch), stream);
}

static int launch_adjoint_fixed(const MarchParams &P, const float *d, const float *t, float *c,
                                const rt_grads &G, cudaStream_t s, float *scr) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return zero_grads(P, G, plan_scratch(P, 1, 0, 0), nullptr, s);
  int LPR, CPL;
  adj_layout(P.nch, &LPR, &CPL);
  const int v = adj_variant(P);
#define X(L, C)                                                           \
  if (LPR == L && CPL == C) {                                             \
    if (v == 0) return launch_adj_fixed_t<L, C, 0>(P, d, t, c, G, s, scr); \
    if (v == 1) return launch_adj_fixed_t<L, C, 1>(P, d, t, c, G, s, scr); \
    if (v == 2) return launch_adj_fixed_t<L, C, 2>(P, d, t, c, G, s, scr); \
    return launch_adj_fixed_t<L, C, 3>(P, d, t, c, G, s, scr);            \
  }
  RTB_ADJ_LAYOUTS(X)
#undef X
  return set_error(RT_EINVAL, "no adjoint layout for %d channels", P.nch);
}

}  // namespace rtb

// Same contract as rt_render_adjoint, without any allocation (see rt.h).
extern "C" int rt_render_adjoint_noalloc(const rt_grid *grid, const rt_fields *fields,
                                         const rt_geom *geom, const rt_view *view,
                                         const rt_line *line, const float *dL_dcube,
                                         const float *target, float *cube_out,
                                         const rt_grads *grads, void *stream) {
  using namespace rtb;
  MarchParams P;  // on the stack: no host allocation either
  int rc = build_params(grid, fields, geom, view, line, &P);
  if (rc == RT_OK) rc = check_adjoint_args(P, dL_dcube, target, grads);
  float *scratch = nullptr;
  if (rc == RT_OK) rc = fixed_scratch_address(&scratch);
  if (rc == RT_OK)
    rc = launch_adjoint_fixed(P, dL_dcube, target, cube_out, *grads, (cudaStream_t)stream,
                              scratch);
  if (rc == RT_OK) clear_error();
  return rc;
}
