// Fused adjoint of the march: forward march with optical-depth checkpoints, then a reverse
// march that recomputes the transmittance and propagates dL/dcube back to every node of the
// (r, z/r) fields and the CO surfaces.
//
// Reverse recursion (per channel; T_k transmittance before sample k, e_k = 2^-dt_k its
// factor over the segment, S_k the source, gI = dL/dI, g = dL/dT_{k+1} from the later part
// of the ray, seeded with dL/dcube * I0 at the far end):
//   G      = g - gI S_k                      full dL/dT_{k+1} (T_{k+1} also enters step k)
//   dL/dS_k  = gI T_k (1 - e_k)
//   dL/ddt_k = -ln2 G T_{k+1}                (dt in log2 units)
//   g     <- g - G (1 - e_k)                 (= G e_k + gI S_k: a convex update, no division)
// with 1 - e_k from a series for small dt (no cancellation). The reverse march runs over
// 64-sample segments from the last to the first: each segment's optical depth at its start
// was checkpointed by the forward pass (device scratch); the batch starts inside the segment
// are recomputed forward into shared memory; the batches are then walked backward, the
// transmittance being rebuilt from the batch-end optical depth by subtracting the recomputed
// per-sample increments.
//
// Per sample, the per-channel partial derivatives (w.r.t. the optical-depth factor kd, the
// profile terms a and b and the source S) are summed over the lanes of the ray through
// shared memory; lane q then applies the chain rule through the sample physics (line width,
// LTE table, Planck source, CO-layer logistic edges, bilinear weights) and scatters the node
// gradients with FP64 atomics.
#include <mutex>

#include "rt_internal.cuh"

namespace rtb {

constexpr int kWarpsAdj = 2;  // warps per block
constexpr int kSeg = 64;      // samples per checkpoint segment
constexpr float kLn2 = 0.6931471805599453f;

// 1 - 2^-x for x >= 0 without cancellation: series of 1 - e^-y (y = x ln 2) up to y^4 below
// y = 0.05 (relative truncation < 6e-8), 1 - ex2(-x) above.
__device__ __forceinline__ float one_minus_ex2neg(float x) {
  if (x < 0.0721347520f)
    return x * fmaf(x, fmaf(x, fmaf(x, -0.00961812910762848f, 0.0555041086648216f),
                            -0.240226506959101f),
                    0.693147180559945f);
  return 1.0f - ex2(-x);
}

// Chain rule of one sample: given dL/dkd, dL/da, dL/db and dL/dS of sample k of ray R,
// accumulate dL/d(node values) with FP64 atomics.
__device__ __forceinline__ void sample_grad(const MarchParams &P, const float *tab, const Ray &R,
                                            int k, float gkd, float ga, float gb, float gS,
                                            const rt_grads &G) {
  float kf = (float)k;
  float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  float r2 = fmaf(R.x, R.x, y * y);
  Cell c = locate(P, z, r2);
  if (!(c.gas && R.hit && k < P.n_samples)) return;
  float T = bilerp(P.T, P.nr, c);
  float n = bilerp(P.n, P.nr, c);
  float vt = bilerp(P.vt, P.nr, c);
  const float *hl = P.hlo + c.i0;
  const float *hh = P.hhi + c.i0;
  float hlo = lerpf(__ldg(hl), __ldg(hl + 1), c.fr);
  float hhi = lerpf(__ldg(hh), __ldg(hh + 1), c.fr);
  float X, dX_dhlo = 0.0f, dX_dhhi = 0.0f;
  if (P.hard_edge) {
    X = (c.zr >= hlo && c.zr <= hhi) ? P.x_co : 0.0f;
  } else {
    float ea = ex2((hlo - c.zr) * P.edge_k);
    float eb = ex2((c.zr - hhi) * P.edge_k);
    float ia_ = rcp(1.0f + ea), ib_ = rcp(1.0f + eb);
    X = P.x_co * ia_ * ib_;
    // X = x_co / ((1 + ea)(1 + eb)), ea = 2^{(hlo - z/r) k}, eb = 2^{(z/r - hhi) k}
    dX_dhlo = -X * (ea * ia_) * P.edge_k * kLn2;
    dX_dhhi = X * (eb * ib_) * P.edge_k * kLn2;
  }
  float vlos = fmaf(R.vfac, kepler_q(fmaf(z, z, r2)), P.vsys);
  bool clampT = T < 1e-3f;
  float Tg = fmaxf(T, 1e-3f);
  float a2 = P.vturb_mach ? Tg * fmaf(P.c_mach, vt * vt, P.c_th) : fmaf(P.c_th, Tg, vt * vt);
  float ia = rsq(a2);
  float dphi;
  float phi = lte_phi(tab, lg2(Tg), &dphi);
  float iT = rcp(Tg);
  float eS = ex2(-P.theta_s * iT);
  float F = ex2(phi);
  const float cb = 1.2011224087864498f;  // b = cb ia, a = vlos b
  // kd = kappa X n F ia ds
  float base = P.kappa_k * F * R.ds;      // kd / (X n ia)
  float kd = base * X * n * ia;
  float g_ia = gkd * base * X * n + (gb + ga * vlos) * cb;
  float g_a2 = g_ia * (-0.5f * ia * ia * ia);
  float dT = 0.0f, dvt;
  if (P.vturb_mach) {
    dT = g_a2 * fmaf(P.c_mach, vt * vt, P.c_th);
    dvt = g_a2 * Tg * P.c_mach * 2.0f * vt;
  } else {
    dT = g_a2 * P.c_th;
    dvt = g_a2 * 2.0f * vt;
  }
  // d 2^Phi(log2 T) / dT = 2^Phi Phi'(t) / T
  dT += gkd * kd * dphi * iT;
  // S = eS / (1 - eS), eS = 2^{-theta/T}: dS/dT = eS ln2 theta / (T^2 (1 - eS)^2)
  float om = rcp(1.0f - eS);
  dT += gS * eS * om * om * kLn2 * P.theta_s * iT * iT;
  if (clampT) dT = 0.0f;
  float dn = gkd * base * X * ia;
  float dX = gkd * base * n * ia;
  float dhlo = dX * dX_dhlo, dhhi = dX * dX_dhhi;
  // bilinear scatter
  int nr = P.nr;
  int i00 = c.j0 * nr + c.i0;
  float w00 = (1.0f - c.fr) * (1.0f - c.fz), w01 = c.fr * (1.0f - c.fz);
  float w10 = (1.0f - c.fr) * c.fz, w11 = c.fr * c.fz;
  int idx[4] = {i00, i00 + 1, i00 + nr, i00 + nr + 1};
  float w[4] = {w00, w01, w10, w11};
#pragma unroll
  for (int a = 0; a < 4; a++) {
    atomicAdd(G.dT + idx[a], (double)(dT * w[a]));
    atomicAdd(G.dn + idx[a], (double)(dn * w[a]));
    atomicAdd(G.dvt + idx[a], (double)(dvt * w[a]));
  }
  atomicAdd(G.dh_lo + c.i0, (double)(dhlo * (1.0f - c.fr)));
  atomicAdd(G.dh_lo + c.i0 + 1, (double)(dhlo * c.fr));
  atomicAdd(G.dh_hi + c.i0, (double)(dhhi * (1.0f - c.fr)));
  atomicAdd(G.dh_hi + c.i0 + 1, (double)(dhhi * c.fr));
}

template <int LPR, int CPL, bool UNIF>
__global__ void __launch_bounds__(kWarpsAdj * 32)
    march_adj_kernel(const __grid_constant__ MarchParams P, const float *__restrict__ dLdc,
                     const float *__restrict__ target, float *__restrict__ cube_out,
                     const rt_grads G, float *__restrict__ scratch, int nseg) {
  constexpr int R = 32 / LPR;
  constexpr int NG = 32 / R;           // work units whose setups are computed together
  constexpr int NB = kSeg / LPR;       // batches per segment
  __shared__ __align__(16) float s_tab[kTabSeg * 4];
  __shared__ float4 s_ph[kWarpsAdj][32];
  __shared__ Ray s_ray[kWarpsAdj][32];
  __shared__ float4 s_part[kWarpsAdj][LPR][32];
  __shared__ float s_tbb[kWarpsAdj][NB + 1][CPL][32];
  for (int i = threadIdx.x; i < kTabSeg * 4; i += blockDim.x) s_tab[i] = P.tab[i];
  __syncthreads();

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = lane % LPR, rr = lane / LPR;
  const long long npix = (long long)P.nx * P.ny;
  const long long nunits = (npix + R - 1) / R;
  const long long W = (long long)gridDim.x * kWarpsAdj;
  const long long gw = (long long)blockIdx.x * kWarpsAdj + wib;
  float *ck = scratch + gw * (long long)nseg * CPL * 32;  // this warp's checkpoints
  float4 *ph = s_ph[wib];
  float vc[CPL];
#pragma unroll
  for (int j = 0; j < CPL; j++)
    vc[j] = UNIF ? fmaf((float)(q + LPR * j), P.dv, P.v0) : P.v[min(q + LPR * j, RT_MAX_CH - 1)];
  const float vq = P.v0 + (float)q * P.dv;
  const float dvs = (float)LPR * P.dv;
  double loss = 0.0;

  for (long long u0 = gw; u0 < nunits; u0 += W * NG) {
    {
      long long pix = (u0 + (long long)(lane / R) * W) * R + lane % R;
      bool act = pix < npix;
      Ray s = setup_ray(P, act ? (int)(pix % P.nx) : 0, act ? (int)(pix / P.nx) : 0, act);
      __syncwarp();
      s_ray[wib][lane] = s;
      __syncwarp();
    }
    for (int gi = 0; gi < NG; gi++) {
      const long long u = u0 + (long long)gi * W;
      if (u >= nunits) break;
      const long long pix = u * R + rr;
      const bool active = pix < npix;
      const Ray ray = s_ray[wib][gi * R + rr];
      const int nsamp = __any_sync(0xffffffffu, ray.hit) ? P.n_samples : 0;

      // ---------------- forward march with checkpoints every kSeg samples ----------------
      float tl[CPL], tb[CPL], Tr[CPL], I[CPL];
#pragma unroll
      for (int j = 0; j < CPL; j++) {
        tl[j] = 0.0f;
        tb[j] = 0.0f;
        Tr[j] = 1.0f;
        I[j] = 0.0f;
      }
      for (int kb = 0; kb < nsamp; kb += LPR) {
        if (kb % kSeg == 0) {
#pragma unroll
          for (int j = 0; j < CPL; j++) ck[((kb / kSeg) * CPL + j) * 32 + lane] = tb[j];
        }
        const float4 mine = sample_physics(P, s_tab, ray, kb + q);
        if (!__any_sync(0xffffffffu, mine.x > 0.0f)) continue;
        ph[lane] = mine;
        __syncwarp();
#pragma unroll
        for (int t = 0; t < LPR; t++) {
          const float4 p = ph[rr * LPR + t];
          const float dc = fmaf(vq, p.z, -p.y), db = dvs * p.z;
#pragma unroll
          for (int j = 0; j < CPL; j++) {
            float d = UNIF ? fmaf((float)j, db, dc) : fmaf(vc[j], p.z, -p.y);
            tl[j] = fmaf(p.x, ex2(d * -d), tl[j]);
            float Tn = ex2(-tb[j] - tl[j]);
            I[j] = fmaf(p.w, Tr[j] - Tn, I[j]);
            Tr[j] = Tn;
          }
        }
#pragma unroll
        for (int j = 0; j < CPL; j++) {
          tb[j] += tl[j];
          tl[j] = 0.0f;
        }
        __syncwarp();
      }

      // ---------------- loss seed ----------------
      float gI[CPL], g[CPL];
#pragma unroll
      for (int j = 0; j < CPL; j++) {
        const int ch = q + LPR * j;
        float go = 0.0f;
        if (active && ch < P.nch) {
          const long long o = (long long)ch * npix + pix;
          const float out = fmaf(I[j], P.out_scale, P.I0 * Tr[j]);
          if (cube_out) cube_out[o] = out;
          if (dLdc) {
            go = dLdc[o];
          } else {
            const float r = out - target[o];
            go = 2.0f * r;
            loss += (double)r * (double)r;
          }
        }
        gI[j] = go * P.out_scale;  // dL/d(internal intensity)
        g[j] = go * P.I0;          // dL/dT at the far end (background term)
      }
      if (nsamp == 0) continue;

      // ---------------- reverse march over segments ----------------
      const int nseg_ray = (P.n_samples + kSeg - 1) / kSeg;
      for (int seg = nseg_ray - 1; seg >= 0; seg--) {
        const int k0 = seg * kSeg;
        const int nb = min(NB, (P.n_samples - k0 + LPR - 1) / LPR);
        // forward recompute of the batch starts of this segment
        float tbs[CPL];
#pragma unroll
        for (int j = 0; j < CPL; j++) tbs[j] = ck[(seg * CPL + j) * 32 + lane];
        for (int b = 0; b < nb; b++) {
#pragma unroll
          for (int j = 0; j < CPL; j++) s_tbb[wib][b][j][lane] = tbs[j];
          const float4 mine = sample_physics(P, s_tab, ray, k0 + b * LPR + q);
          if (!__any_sync(0xffffffffu, mine.x > 0.0f)) continue;
          ph[lane] = mine;
          __syncwarp();
          float ts[CPL];
#pragma unroll
          for (int j = 0; j < CPL; j++) ts[j] = 0.0f;
#pragma unroll
          for (int t = 0; t < LPR; t++) {
            const float4 p = ph[rr * LPR + t];
            const float dc = fmaf(vq, p.z, -p.y), db = dvs * p.z;
#pragma unroll
            for (int j = 0; j < CPL; j++) {
              float d = UNIF ? fmaf((float)j, db, dc) : fmaf(vc[j], p.z, -p.y);
              ts[j] = fmaf(p.x, ex2(d * -d), ts[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < CPL; j++) tbs[j] += ts[j];
          __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < CPL; j++) s_tbb[wib][nb][j][lane] = tbs[j];
        __syncwarp();

        // backward over the batches of the segment
        for (int b = nb - 1; b >= 0; b--) {
          const int kb = k0 + b * LPR;
          const float4 mine = sample_physics(P, s_tab, ray, kb + q);
          if (!__any_sync(0xffffffffu, mine.x > 0.0f)) continue;  // identity batch
          ph[lane] = mine;
          float cur[CPL], Tn[CPL];
#pragma unroll
          for (int j = 0; j < CPL; j++) {
            cur[j] = s_tbb[wib][b + 1][j][lane];
            Tn[j] = ex2(-cur[j]);
          }
          __syncwarp();
#pragma unroll
          for (int t = LPR - 1; t >= 0; t--) {
            const float4 p = ph[rr * LPR + t];
            const float dc = fmaf(vq, p.z, -p.y), db = dvs * p.z;
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < CPL; j++) {
              const float d = UNIF ? fmaf((float)j, db, dc) : fmaf(vc[j], p.z, -p.y);
              const float gg = ex2(d * -d);
              const float dt = p.x * gg;
              cur[j] -= dt;
              const float T0 = ex2(-cur[j]);
              const float om = one_minus_ex2neg(dt);
              const float Gf = g[j] - gI[j] * p.w;
              const float dtl = -kLn2 * Gf * Tn[j];  // dL/d dt
              acc.w = fmaf(gI[j] * T0, om, acc.w);   // dL/dS
              g[j] = fmaf(-Gf, om, g[j]);
              Tn[j] = T0;
              acc.x = fmaf(dtl, gg, acc.x);          // dL/dkd
              const float dd = dtl * dt * (-2.0f * kLn2) * d;  // dL/dd
              acc.y -= dd;                           // d = v b - a
              acc.z = fmaf(dd, vc[j], acc.z);
            }
            s_part[wib][t][lane] = acc;
          }
          __syncwarp();
          // sum the partials of sample kb+q over the lanes of this ray, then the chain rule
          float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
          for (int i = 0; i < LPR; i++) {
            const float4 v = s_part[wib][q][rr * LPR + i];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
          }
          if (active && mine.x > 0.0f) sample_grad(P, s_tab, ray, kb + q, s.x, s.y, s.z, s.w, G);
          __syncwarp();
        }
      }
    }
  }
  if (G.loss && target) {
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if (lane == 0 && loss != 0.0) atomicAdd(G.loss, loss);
  }
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

// Launch geometry of the adjoint kernel for P: blocks of the persistent grid and the
// checkpoint scratch they need. cap_blocks <= 0 asks the occupancy calculator.
template <int LPR, int CPL, bool UNIF>
static void adj_geometry(const MarchParams &P, long long cap_blocks, long long *blocks,
                         size_t *bytes) {
  long long npix = (long long)P.nx * P.ny;
  long long units = (npix + (32 / LPR) - 1) / (32 / LPR);
  long long need = (units + kWarpsAdj - 1) / kWarpsAdj;
  long long cap = cap_blocks > 0
                      ? cap_blocks
                      : resident_blocks((const void *)march_adj_kernel<LPR, CPL, UNIF>,
                                        kWarpsAdj * 32);
  *blocks = need < cap ? need : cap;
  int nseg = (P.n_samples + kSeg - 1) / kSeg;
  *bytes = (size_t)(*blocks) * kWarpsAdj * nseg * CPL * 32 * sizeof(float);
}

template <int LPR, int CPL, bool UNIF>
static int launch_adj_t(const MarchParams &P, const float *dLdc, const float *target,
                        float *cube_out, const rt_grads &G, cudaStream_t stream) {
  auto kern = march_adj_kernel<LPR, CPL, UNIF>;
  long long blocks;
  size_t bytes;
  adj_geometry<LPR, CPL, UNIF>(P, 0, &blocks, &bytes);
  int nseg = (P.n_samples + kSeg - 1) / kSeg;
  float *scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&scratch, bytes, stream);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "adjoint scratch (%zu bytes): %s", bytes, cudaGetErrorString(e));
  kern<<<(unsigned)blocks, kWarpsAdj * 32, 0, stream>>>(P, dLdc, target, cube_out, G, scratch,
                                                         nseg);
  e = cudaGetLastError();
  cudaFreeAsync(scratch, stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "adjoint launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

template <int LPR, int CPL>
static int launch_adj_u(const MarchParams &P, const float *dLdc, const float *target,
                        float *cube_out, const rt_grads &G, cudaStream_t s) {
  return P.v_uniform ? launch_adj_t<LPR, CPL, true>(P, dLdc, target, cube_out, G, s)
                     : launch_adj_t<LPR, CPL, false>(P, dLdc, target, cube_out, G, s);
}

// Zeroes the gradient outputs and launches the fused adjoint.
int launch_adjoint(const MarchParams &P, const float *dLdc, const float *target,
                   float *cube_out, const rt_grads &G, cudaStream_t stream) {
  size_t ng = (size_t)P.nr * P.nz * sizeof(double), nh = (size_t)P.nr * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dT, 0, ng, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dn, 0, ng, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dvt, 0, ng, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dh_lo, 0, nh, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dh_hi, 0, nh, stream);
  if (e == cudaSuccess && G.loss) e = cudaMemsetAsync(G.loss, 0, sizeof(double), stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "gradient memset: %s", cudaGetErrorString(e));
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return RT_OK;
  int LPR, CPL;
  lane_layout(P.nch, &LPR, &CPL);
  const float *d = dLdc;
  const float *t = target;
  if (CPL == 8) return launch_adj_u<32, 8>(P, d, t, cube_out, G, stream);
  if (LPR == 32) return launch_adj_u<32, 4>(P, d, t, cube_out, G, stream);
  if (LPR == 16) return launch_adj_u<16, 4>(P, d, t, cube_out, G, stream);
  if (LPR == 8) return launch_adj_u<8, 4>(P, d, t, cube_out, G, stream);
  if (LPR == 4) return launch_adj_u<4, 4>(P, d, t, cube_out, G, stream);
  if (LPR == 2) return launch_adj_u<2, 4>(P, d, t, cube_out, G, stream);
  // one lane per ray would need 65 batch starts per warp in shared memory: use two
  return launch_adj_u<2, 4>(P, d, t, cube_out, G, stream);
}

// Checkpoint scratch rt_render_adjoint allocates for P (cap_blocks > 0 replaces the device
// occupancy query, for planning without a GPU).
size_t adjoint_scratch_bytes(const MarchParams &P, long long cap_blocks) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return 0;
  int LPR, CPL;
  lane_layout(P.nch, &LPR, &CPL);
  long long b;
  size_t bytes = 0;
  const bool u = P.v_uniform != 0;
#define RTB_GEOM(L, C)                                               \
  (u ? adj_geometry<L, C, true>(P, cap_blocks, &b, &bytes)           \
     : adj_geometry<L, C, false>(P, cap_blocks, &b, &bytes))
  if (CPL == 8) RTB_GEOM(32, 8);
  else if (LPR == 32) RTB_GEOM(32, 4);
  else if (LPR == 16) RTB_GEOM(16, 4);
  else if (LPR == 8) RTB_GEOM(8, 4);
  else if (LPR == 4) RTB_GEOM(4, 4);
  else RTB_GEOM(2, 4);
#undef RTB_GEOM
  return bytes;
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
// is running. For them the checkpoint scratch of the adjoint lives in one file-scope device
// array of fixed size, kFixedScratchBytes, that every GPU loading this library holds until
// the process exits. The kernel is the same; when the array cannot hold a checkpoint region
// for every resident block, the persistent grid is made smaller (same result, lower
// throughput), and a problem that does not fit even one block is rejected.
// ---------------------------------------------------------------------------------------
namespace rtb {

constexpr size_t kFixedScratchBytes = (size_t)16 << 20;  // 16 MiB per device
static __device__ __align__(256) float g_fixed_scratch[kFixedScratchBytes / sizeof(float)];

// Device address of g_fixed_scratch on the current device. The host-side name is only a
// stand-in for the symbol, so the address is looked up once per device (with that device
// current) and cached.
static int fixed_scratch_address(float **out) {
  static std::mutex mu;
  static float *addr[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(RT_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fixed_scratch);
    if (e != cudaSuccess || !p)
      return set_error(RT_ECUDA, "cudaGetSymbolAddress(fixed scratch): %s", cudaGetErrorString(e));
    addr[dev] = (float *)p;
  }
  *out = addr[dev];
  return RT_OK;
}

template <int LPR, int CPL, bool UNIF>
static int launch_adj_fixed_t(const MarchParams &P, const float *dLdc, const float *target,
                              float *cube_out, const rt_grads &G, cudaStream_t stream,
                              float *scratch) {
  auto kern = march_adj_kernel<LPR, CPL, UNIF>;
  long long npix = (long long)P.nx * P.ny;
  long long units = (npix + (32 / LPR) - 1) / (32 / LPR);
  long long need = (units + kWarpsAdj - 1) / kWarpsAdj;
  long long cap = resident_blocks((const void *)kern, kWarpsAdj * 32);
  int nseg = (P.n_samples + kSeg - 1) / kSeg;
  size_t per_block = (size_t)kWarpsAdj * nseg * CPL * 32 * sizeof(float);
  if (per_block > kFixedScratchBytes)
    return set_error(RT_EINVAL,
                     "allocation-free adjoint: %d samples per ray need %zu bytes of checkpoint "
                     "scratch per block, above the fixed %zu-byte array",
                     P.n_samples, per_block, kFixedScratchBytes);
  long long fit = (long long)(kFixedScratchBytes / per_block);
  long long blocks = need < cap ? need : cap;
  if (blocks > fit) blocks = fit;
  kern<<<(unsigned)blocks, kWarpsAdj * 32, 0, stream>>>(P, dLdc, target, cube_out, G, scratch,
                                                         nseg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "adjoint launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

template <int LPR, int CPL>
static int launch_adj_fixed_u(const MarchParams &P, const float *d, const float *t, float *c,
                              const rt_grads &G, cudaStream_t s, float *scr) {
  return P.v_uniform ? launch_adj_fixed_t<LPR, CPL, true>(P, d, t, c, G, s, scr)
                     : launch_adj_fixed_t<LPR, CPL, false>(P, d, t, c, G, s, scr);
}

static int launch_adjoint_fixed(const MarchParams &P, const float *d, const float *t, float *c,
                                const rt_grads &G, cudaStream_t s, float *scr) {
  size_t ng = (size_t)P.nr * P.nz * sizeof(double), nh = (size_t)P.nr * sizeof(double);
  cudaError_t e = cudaMemsetAsync(G.dT, 0, ng, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dn, 0, ng, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dvt, 0, ng, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dh_lo, 0, nh, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.dh_hi, 0, nh, s);
  if (e == cudaSuccess && G.loss) e = cudaMemsetAsync(G.loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "gradient memset: %s", cudaGetErrorString(e));
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return RT_OK;
  int LPR, CPL;
  lane_layout(P.nch, &LPR, &CPL);
  if (CPL == 8) return launch_adj_fixed_u<32, 8>(P, d, t, c, G, s, scr);
  if (LPR == 32) return launch_adj_fixed_u<32, 4>(P, d, t, c, G, s, scr);
  if (LPR == 16) return launch_adj_fixed_u<16, 4>(P, d, t, c, G, s, scr);
  if (LPR == 8) return launch_adj_fixed_u<8, 4>(P, d, t, c, G, s, scr);
  if (LPR == 4) return launch_adj_fixed_u<4, 4>(P, d, t, c, G, s, scr);
  return launch_adj_fixed_u<2, 4>(P, d, t, c, G, s, scr);
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
