// Forward march kernel.
//
// Mapping: a warp owns a tile of kTileRays consecutive pixels. Their ray setups (double
// precision chord through the bounding cylinder) are computed once, one lane per ray, and
// kept in shared memory. The warp then marches R = 32/LPR rays at a time: the LPR lanes of a
// ray split its channels (lane q holds channels q, q+LPR, q+2 LPR, ... in registers).
// Samples advance in batches of LPR: in the physics phase lane q evaluates the
// channel-independent physics of sample kb+q of its ray (fields, CO layer, Keplerian
// velocity, line width, LTE source and opacity) once and publishes it in shared memory; in
// the channel phase every lane walks, in order and four at a time, the batch's samples that
// carry gas (warp ballot), evaluating the Doppler-shifted Gaussian profile and advancing
// optical depth, transmittance and intensity front to back (Eq. rt-int with
// Eq. optical_depth; the source is constant over each segment).
//
// Per sample-channel evaluation: 7 FP32 operations and 2 MUFU.EX2. The optical depth is
// summed per batch and folded into a per-channel base at the end of every batch (blocked
// summation: about 2 N_s / LPR roundings instead of N_s).
#include "rt_internal.cuh"

namespace rtb {

constexpr int kWarps = 4;      // warps per block
constexpr int kTileRays = 8;   // rays per warp tile

// Channel-independent physics of sample k of a ray: {kd, a, b, S} with
//   kd  optical depth per unit profile (log2 units): dtau_c = kd 2^{-d_c^2}, 0 without gas
//   a,b profile argument d_c = v_c b - a (b = sqrt(log2 e)/alpha, a = v_los b)
//   S   LTE source function in units of 2 h nu0^3 / c^2
__device__ __forceinline__ float4 sample_physics(const MarchParams &P, const float *tab,
                                                 const Ray &R, int k) {
  float kf = (float)k;
  float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  float r2 = fmaf(R.x, R.x, y * y);
  Cell c = locate(P, z, r2);
  float4 out = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  if (!(c.gas && R.hit && k < P.n_samples)) return out;
  float T = bilerp(P.T, P.nr, c);
  float n = bilerp(P.n, P.nr, c);
  float vt = bilerp(P.vt, P.nr, c);
  const float *hl = P.hlo + c.i0;
  const float *hh = P.hhi + c.i0;
  float hlo = lerpf(__ldg(hl), __ldg(hl + 1), c.fr);
  float hhi = lerpf(__ldg(hh), __ldg(hh + 1), c.fr);
  float X;
  if (P.hard_edge) {
    X = (c.zr >= hlo && c.zr <= hhi) ? P.x_co : 0.0f;
  } else {
    float ea = ex2((hlo - c.zr) * P.edge_k);
    float eb = ex2((c.zr - hhi) * P.edge_k);
    X = P.x_co * rcp((1.0f + ea) * (1.0f + eb));
  }
  // Keplerian rotation: v_los = sqrt(GM) sin i x (r^2 + z^2)^{-3/4} + v_sys
  float vlos = fmaf(R.vfac, kepler_q(fmaf(z, z, r2)), P.vsys);
  // line width
  float Tg = fmaxf(T, 1e-3f);
  float a2 = P.vturb_mach ? Tg * fmaf(P.c_mach, vt * vt, P.c_th) : fmaf(P.c_th, Tg, vt * vt);
  float ia = rsq(a2);
  // LTE: source function and tabulated lower-level opacity factor
  float phi = lte_phi(tab, lg2(Tg), nullptr);
  float eS = ex2(-P.theta_s * rcp(Tg));
  out.w = eS * rcp(1.0f - eS);
  out.x = P.kappa_k * (X * n) * ex2(phi) * ia * R.ds;
  out.z = ia * 1.2011224087864498f;  // b = sqrt(log2 e) / alpha
  out.y = vlos * out.z;              // a = v_los b
  return out;
}

template <int LPR, int CPL, bool UNIF>
__global__ void __launch_bounds__(kWarps * 32)
    march_fwd_kernel(const __grid_constant__ MarchParams P, float *__restrict__ cube) {
  constexpr int R = 32 / LPR;  // rays marched together by one warp
  __shared__ __align__(16) float s_tab[kTabSeg * 4];
  __shared__ float4 s_ph[kWarps][32];
  __shared__ Ray s_ray[kWarps][kTileRays];
  for (int i = threadIdx.x; i < kTabSeg * 4; i += blockDim.x) s_tab[i] = P.tab[i];

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = lane % LPR, rr = lane / LPR;
  const long long npix = (long long)P.nx * P.ny;
  const long long tile0 = ((long long)blockIdx.x * kWarps + wib) * kTileRays;
  if (lane < kTileRays) {
    long long pix = tile0 + lane;
    bool act = pix < npix;
    s_ray[wib][lane] = setup_ray(P, act ? (int)(pix % P.nx) : 0, act ? (int)(pix / P.nx) : 0, act);
  }
  __syncthreads();
  float4 *ph = s_ph[wib];

  float vr[UNIF ? 1 : CPL];
  if (!UNIF) {
#pragma unroll
    for (int j = 0; j < CPL; j++) vr[j] = P.v[min(q + LPR * j, RT_MAX_CH - 1)];
  }
  const float vq = P.v0 + (float)q * P.dv;  // velocity of this lane's first channel
  const float dvs = (float)LPR * P.dv;      // spacing between this lane's channels

  for (int it = 0; it < kTileRays / R; it++) {
    const int ri = it * R + rr;
    const long long pix = tile0 + ri;
    const Ray ray = s_ray[wib][ri];
    float tl[CPL], tb[CPL], Tr[CPL], I[CPL];
#pragma unroll
    for (int j = 0; j < CPL; j++) {
      tl[j] = 0.0f;
      tb[j] = 0.0f;
      Tr[j] = 1.0f;
      I[j] = 0.0f;
    }
    const int nsamp = __any_sync(0xffffffffu, ray.hit) ? P.n_samples : 0;
    for (int kb = 0; kb < nsamp; kb += LPR) {
      float4 mine = sample_physics(P, s_tab, ray, kb + q);
      unsigned gm = __ballot_sync(0xffffffffu, mine.x > 0.0f);
      if (gm == 0u) continue;  // no gas in this batch on any ray of the warp
      ph[lane] = mine;
      __syncwarp();
      unsigned m = gm;
#pragma unroll
      for (int s = 1; s < R; s++) m |= gm >> (s * LPR);
      if (LPR < 32) m &= (1u << (LPR & 31)) - 1u;
      while (m) {
        // next four gas samples (in order); missing ones are exact no-ops (kd = 0)
        float4 p[4];
        float dc[4], db[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          int t = __ffs(m) - 1;
          m &= m - 1;
          p[u] = t >= 0 ? ph[rr * LPR + t] : make_float4(0.0f, 0.0f, 1.0f, 0.0f);
          dc[u] = fmaf(vq, p[u].z, -p[u].y);
          db[u] = dvs * p[u].z;
        }
#pragma unroll
        for (int j = 0; j < CPL; j++) {
          float dt[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            float d = UNIF ? fmaf((float)j, db[u], dc[u]) : fmaf(vr[j], p[u].z, -p[u].y);
            dt[u] = p[u].x * ex2(d * -d);
          }
#pragma unroll
          for (int u = 0; u < 4; u++) {
            tl[j] += dt[u];
            float Tn = ex2(-tb[j] - tl[j]);
            I[j] = fmaf(p[u].w, Tr[j] - Tn, I[j]);
            Tr[j] = Tn;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < CPL; j++) {
        tb[j] += tl[j];
        tl[j] = 0.0f;
      }
      __syncwarp();
    }
    if (pix < npix) {
#pragma unroll
      for (int j = 0; j < CPL; j++) {
        int ch = q + LPR * j;
        if (ch < P.nch) cube[(long long)ch * npix + pix] = fmaf(I[j], P.out_scale, P.I0 * Tr[j]);
      }
    }
  }
}

template <int LPR, int CPL>
static void launch_t(const MarchParams &P, float *cube, cudaStream_t stream, unsigned blocks) {
  if (P.v_uniform)
    march_fwd_kernel<LPR, CPL, true><<<blocks, kWarps * 32, 0, stream>>>(P, cube);
  else
    march_fwd_kernel<LPR, CPL, false><<<blocks, kWarps * 32, 0, stream>>>(P, cube);
}

int launch_forward(const MarchParams &P, float *cube, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return RT_OK;
  int LPR = P.nch <= 8 ? 8 : (P.nch <= 16 ? 16 : 32);
  int CPL = (P.nch + LPR - 1) / LPR;
  long long per_block = (long long)kWarps * kTileRays;
  long long blocks = (npix + per_block - 1) / per_block;
  if (blocks > 0x7fffffffLL) return set_error(RT_EINVAL, "image too large");
  unsigned b = (unsigned)blocks;
  if (LPR == 8) launch_t<8, 1>(P, cube, stream, b);
  else if (LPR == 16) launch_t<16, 1>(P, cube, stream, b);
  else if (CPL == 1) launch_t<32, 1>(P, cube, stream, b);
  else if (CPL == 2) launch_t<32, 2>(P, cube, stream, b);
  else if (CPL <= 4) launch_t<32, 4>(P, cube, stream, b);
  else launch_t<32, 8>(P, cube, stream, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "forward launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

// Work count: (ray, sample) pairs of hit rays that fall inside the gas grid, i.e. the
// executed (rather than nominal) samples of a render.
__global__ void count_gas_kernel(const __grid_constant__ MarchParams P,
                                 unsigned long long *__restrict__ count) {
  const long long npix = (long long)P.nx * P.ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long n = 0;
  if (pix < npix) {
    Ray R = setup_ray(P, (int)(pix % P.nx), (int)(pix / P.nx), true);
    if (R.hit) {
      for (int k = 0; k < P.n_samples; k++) {
        float kf = (float)k;
        float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
        float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
        Cell c = locate(P, z, fmaf(R.x, R.x, y * y));
        n += c.gas ? 1 : 0;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, n);
}

int launch_count(const MarchParams &P, unsigned long long *count, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "count memset: %s", cudaGetErrorString(e));
  if (npix == 0) return RT_OK;
  long long blocks = (npix + 255) / 256;
  count_gas_kernel<<<(unsigned)blocks, 256, 0, stream>>>(P, count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "count launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rtb
