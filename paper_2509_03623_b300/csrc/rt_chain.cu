// Physics-constrained field chain (arXiv 2509.03623, Methods: "Parametric Disk Modeling",
// Eq. gas_density_temp (vertical hydrostatic equilibrium), the surface-density profile
// Sigma(r), Eq. column_density (H2 column above a point) and Eq. co_layer (freeze-out and
// photodissociation); "Neural Temperature Recovery" derives these secondary fields from the
// temperature, so this is the step that turns a temperature grid into the density and CO
// layer the march reads).
//
// Per radius node r_i, on the node heights z_j = w_j r_i (w_j = j zr_max / (nz - 1)):
//   ln rho_j = ln rho_0 - I_j - ln(T_j / T_0),  I_j = int_0^{z_j} G M m_mol z / ((r^2+z^2)^{3/2} k T) dz
//     (trapezoid rule on the nodes; the d ln T / dz term integrates exactly);
//   rho normalised so that 2 int_0^{z_max} rho dz (trapezoid) = Sigma(r);
//   n_H2 = rho / m_mol;  N_H2(z_j) = int_{z_j}^{z_max} n_H2 dz (trapezoid);
//   the CO layer {T > T_freeze, 0.706 N_H2 > N_dissoc} as two surfaces in z/r: h_lo at the
//   first upward crossing of T_freeze (T linear between nodes), h_hi where 0.706 N_H2 falls to
//   N_dissoc (N_H2 linear between nodes).
//
// One warp per radius column: lanes take 32 consecutive nodes at a time, the two running
// integrals are warp scans (upward for I, downward for N) with a carry between chunks, and
// the surfaces come from warp ballots. FP32 throughout. Pass 1 leaves the unnormalised
// density in n_h2; pass 2 scales it and integrates the column from the top.
#include "rt_internal.cuh"

namespace rtb {

struct ChainDev {
  int nr, nz, r_log;
  float r_in, r_out;
  double zr_max;
  float sigma0, r_c, gamma;
  float A;         // G M m_mol / (k au) [K au]: gravity term per au of height, times 1/T
  float m_mol_g;   // mean molecular mass [g]
  float T_freeze, N_dissoc;
};

constexpr double kChainGMsun = 1.3271244e26;    // cm^3 s^-2
constexpr double kChainK = 1.380649e-16;        // erg / K
constexpr double kChainAmu = 1.66053906660e-24; // g
constexpr double kChainAu = 1.495978707e13;     // cm

__global__ void field_chain_kernel(const ChainDev C, const float *__restrict__ T,
                                   float *__restrict__ n_out, float *__restrict__ N_out,
                                   float *__restrict__ h_lo, float *__restrict__ h_hi) {
  const int lane = threadIdx.x & 31;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= C.nr) return;  // warp-uniform
  const unsigned full = 0xffffffffu;
  const int nr = C.nr, nz = C.nz;
  const int nchunk = (nz + 31) / 32;

  // per-column constants (FP32 library functions, a few ulp: far inside the tolerance)
  const float t = (float)i / (float)(nr - 1);
  const float r = C.r_log ? C.r_in * powf(C.r_out / C.r_in, t) : fmaf(C.r_out - C.r_in, t, C.r_in);
  const float x = r / C.r_c;
  const float sig = C.sigma0 * powf(x, -C.gamma) * expf(-powf(x, 2.0f - C.gamma));
  const float dw = (float)(C.zr_max / (nz - 1));
  const float dz = dw * r;  // au
  const float r2 = r * r;
  const float T0 = __ldg(T + i);

  // ---- pass 1 (upward): I_j, unnormalised density e_j, trapezoid sum, freeze-out crossing ----
  float I_carry = 0.0f, g_carry = 0.0f, S = 0.0f;
  int j_warm = -1;  // first node with T > T_freeze
  for (int c = 0; c < nchunk; c++) {
    const int j = 32 * c + lane;
    const bool valid = j < nz;
    const float Tj = valid ? __ldg(T + (long long)j * nr + i) : 1.0f;
    const float z = dw * (float)j * r;
    const float d = fmaf(z, z, r2);
    const float g = C.A * z / (d * sqrtf(d) * Tj);  // [1/au]
    float gprev = __shfl_up_sync(full, g, 1);
    if (lane == 0) gprev = g_carry;
    float inc = (valid && j > 0) ? 0.5f * dz * (gprev + g) : 0.0f;
    // inclusive warp scan of the trapezoid increments
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float v = __shfl_up_sync(full, inc, o);
      if (lane >= o) inc += v;
    }
    const float I = I_carry + inc;
    const float e = expf(-I - logf(Tj / T0));
    if (valid) {
      n_out[(long long)j * nr + i] = e;
      S += (j == 0 || j == nz - 1) ? 0.5f * e : e;
    }
    I_carry = __shfl_sync(full, I, 31);
    g_carry = __shfl_sync(full, g, 31);
    if (j_warm < 0) {
      const unsigned warm = __ballot_sync(full, valid && Tj > C.T_freeze);
      if (warm) j_warm = 32 * c + __ffs(warm) - 1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(full, S, o);
  S *= dz;  // trapezoid integral of e over [0, z_max] in au

  // freeze-out surface
  if (lane == 0) {
    float lo;
    if (j_warm < 0) {
      lo = (float)C.zr_max;
    } else if (j_warm == 0) {
      lo = 0.0f;
    } else {
      const float Ta = __ldg(T + (long long)(j_warm - 1) * nr + i);
      const float Tb = __ldg(T + (long long)j_warm * nr + i);
      lo = dw * ((float)(j_warm - 1) + (C.T_freeze - Ta) / (Tb - Ta));
    }
    h_lo[i] = lo;
  }

  // ---- pass 2 (downward): n = e * Sigma / (2 S m_mol), column N, photodissociation ----
  __syncwarp();
  const float scale = sig / (2.0f * S * (float)kChainAu * C.m_mol_g);  // [cm^-3] per unit e
  const float dzc = dz * (float)kChainAu;                               // cm
  float N_carry = 0.0f, n_carry = 0.0f;  // N and n at the first node of the chunk above
  bool found = false;
  float hi = 0.0f;
  for (int c = nchunk - 1; c >= 0; c--) {
    const int j = 32 * c + lane;
    const bool valid = j < nz;
    const float n = valid ? n_out[(long long)j * nr + i] * scale : 0.0f;
    if (valid) n_out[(long long)j * nr + i] = n;
    float nnext = __shfl_down_sync(full, n, 1);
    if (lane == 31) nnext = n_carry;
    float seg = (valid && j < nz - 1) ? 0.5f * dzc * (n + nnext) : 0.0f;
    // inclusive suffix scan: seg_j + seg_{j+1} + ... within the chunk
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float v = __shfl_down_sync(full, seg, o);
      if (lane + o < 32) seg += v;
    }
    const float N = N_carry + seg;
    if (valid && N_out) N_out[(long long)j * nr + i] = N;
    if (!found) {
      const unsigned thick = __ballot_sync(full, valid && 0.706f * N > C.N_dissoc);
      if (thick) {
        found = true;
        const int top = 31 - __clz(thick);  // highest qualifying node of the chunk
        float Nb = __shfl_down_sync(full, N, 1);
        if (lane == 31) Nb = N_carry;
        const float Na = __shfl_sync(full, N, top);
        Nb = __shfl_sync(full, Nb, top);
        const float a = 0.706f * Na, b = 0.706f * Nb;
        hi = dw * ((float)(32 * c + top) + (a - C.N_dissoc) / (a - b));
      }
    }
    N_carry = __shfl_sync(full, N, 0);
    n_carry = __shfl_sync(full, n, 0);
  }
  if (lane == 0) h_hi[i] = hi;
}

// ---------------------------------------------------------------------------------------
// Pressure-corrected rotation (Eq. gas_velocity_pressure) on the nodes:
//   v_phi^2 = G M r^2 / (r^2 + z^2)^{3/2} + (r / rho) dP/dr |_z,  P = n k T,  rho = m_mol n,
// dP/dr at constant z from the grid coordinates (u = ln r or r, w = z/r):
//   dP/dr |_z = (du/dr) dP/du |_w - (w / r) dP/dw |_u,
// second-order central differences (second-order one-sided at the first and last node,
// first order on a two-node axis); v_phi^2 < 0 gives 0, a node without gas keeps the
// Keplerian term. One thread per node (a 5-point stencil of n T), FP32 with the
// gravitational term from per-node FP32 geometry; output in km/s.
// ---------------------------------------------------------------------------------------
struct VphiDev {
  int nr, nz, r_log;
  float r_in, r_out;
  float lnratio;  // ln(r_out / r_in)
  float hu, hw;   // node spacings in u (ln r, or r in au) and w
  float gm;       // G M / au [km^2 s^-2]: v^2 = gm r^2 / (r^2+z^2)^{3/2} with r, z in au
  float kpm;      // k / (m_mol) [km^2 s^-2 K^-1]
};

__device__ __forceinline__ float nT_at(const float *__restrict__ n, const float *__restrict__ T,
                                       long long k) {
  return __ldg(n + k) * __ldg(T + k);
}

// derivative of n T along an axis of `cnt` nodes spaced h at node index a (stride s)
__device__ __forceinline__ float axis_d(const float *__restrict__ n, const float *__restrict__ T,
                                        long long base, long long s, int cnt, int a, float h) {
  if (cnt == 2) return (nT_at(n, T, base + s) - nT_at(n, T, base)) / h;
  if (a == 0)
    return (-3.0f * nT_at(n, T, base) + 4.0f * nT_at(n, T, base + s) - nT_at(n, T, base + 2 * s)) /
           (2.0f * h);
  const long long k = base + a * s;
  if (a == cnt - 1)
    return (3.0f * nT_at(n, T, k) - 4.0f * nT_at(n, T, k - s) + nT_at(n, T, k - 2 * s)) / (2.0f * h);
  return (nT_at(n, T, k + s) - nT_at(n, T, k - s)) / (2.0f * h);
}

__global__ void pressure_vphi_kernel(const VphiDev V, const float *__restrict__ n,
                                     const float *__restrict__ T, float *__restrict__ vphi) {
  const long long total = (long long)V.nr * V.nz;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / V.nr), i = (int)(k - (long long)j * V.nr);
    const float t = (float)i / (float)(V.nr - 1);
    const float r = V.r_log ? V.r_in * expf(V.lnratio * t) : fmaf(V.r_out - V.r_in, t, V.r_in);
    const float w = V.hw * (float)j;
    const float d = fmaf(w * w, r * r, r * r);  // r^2 + z^2 [au^2]
    float v2 = V.gm * r * r / (d * sqrtf(d));
    const float nk = __ldg(n + k);
    if (nk > 0.0f) {
      const float dPu = axis_d(n, T, (long long)j * V.nr, 1, V.nr, i, V.hu);
      const float dPw = axis_d(n, T, i, V.nr, V.nz, j, V.hw);
      const float dudr = V.r_log ? 1.0f / r : 1.0f;  // per au
      const float dPdr = fmaf(dudr, dPu, -(w / r) * dPw);  // d(nT)/dr per au
      v2 = fmaf(r / nk, V.kpm * dPdr, v2);
    }
    vphi[k] = v2 > 0.0f ? sqrtf(v2) : 0.0f;
  }
}

int launch_pressure_vphi(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                         const float *n, const float *T, float *vphi, cudaStream_t stream) {
  VphiDev V;
  V.nr = g.nr;
  V.nz = g.nz;
  V.r_log = g.r_log;
  V.r_in = (float)g.r_in_au;
  V.r_out = (float)g.r_out_au;
  V.lnratio = (float)log(g.r_out_au / g.r_in_au);
  V.hu = g.r_log ? (float)(log(g.r_out_au / g.r_in_au) / (g.nr - 1))
                 : (float)((g.r_out_au - g.r_in_au) / (g.nr - 1));
  V.hw = (float)(g.zr_max / (g.nz - 1));
  V.gm = (float)(kChainGMsun * geo.mstar_msun / kChainAu / 1e10);
  V.kpm = (float)(kChainK / (line.m_mol_amu * kChainAmu) / 1e10);
  const long long total = (long long)g.nr * g.nz;
  const long long blocks = (total + 255) / 256;
  pressure_vphi_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(V, n, T,
                                                                                      vphi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "rotation launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

// Reverse mode of the rotation: from dL/dv_phi (per km/s) to dL/dn_H2 and dL/dT. Per node with
// gas and v_phi^2 > 0 (clamped and gas-free nodes contribute nothing): dL/dv^2 = g / (2 v),
//   the direct 1/n term: dL/dn_k += -dL/dv^2 (r / n_k^2) (k/m) dP/dr,
//   the pressure gradient: dL/dQ_l += dL/dv^2 (r / n_k) (k/m) (du/dr c^u_l - (w/r) c^w_l) for the
//   stencil coefficients c of the two differences (Q = n T), scattered with FP64 atomics;
// then dL/dn_l += dL/dQ_l T_l and dL/dT_l = dL/dQ_l n_l.
__device__ __forceinline__ void axis_d_adjoint(double *G, long long base, long long s, int cnt,
                                               int a, float h, float g) {
  if (cnt == 2) {
    atomicAdd(G + base, (double)(-g / h));
    atomicAdd(G + base + s, (double)(g / h));
    return;
  }
  const float c = g / (2.0f * h);
  if (a == 0) {
    atomicAdd(G + base, (double)(-3.0f * c));
    atomicAdd(G + base + s, (double)(4.0f * c));
    atomicAdd(G + base + 2 * s, (double)(-c));
    return;
  }
  const long long k = base + a * s;
  if (a == cnt - 1) {
    atomicAdd(G + k, (double)(3.0f * c));
    atomicAdd(G + k - s, (double)(-4.0f * c));
    atomicAdd(G + k - 2 * s, (double)c);
    return;
  }
  atomicAdd(G + k + s, (double)c);
  atomicAdd(G + k - s, (double)(-c));
}

__global__ void pressure_vphi_adjoint_kernel(const VphiDev V, const float *__restrict__ n,
                                             const float *__restrict__ T,
                                             const double *__restrict__ g_v,
                                             double *__restrict__ g_n, double *gQ) {
  const long long total = (long long)V.nr * V.nz;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / V.nr), i = (int)(k - (long long)j * V.nr);
    const float t = (float)i / (float)(V.nr - 1);
    const float r = V.r_log ? V.r_in * expf(V.lnratio * t) : fmaf(V.r_out - V.r_in, t, V.r_in);
    const float w = V.hw * (float)j;
    const float d = fmaf(w * w, r * r, r * r);
    const float nk = __ldg(n + k);
    double gnk = 0.0;
    if (nk > 0.0f) {
      const float dPu = axis_d(n, T, (long long)j * V.nr, 1, V.nr, i, V.hu);
      const float dPw = axis_d(n, T, i, V.nr, V.nz, j, V.hw);
      const float dudr = V.r_log ? 1.0f / r : 1.0f;
      const float dPdr = fmaf(dudr, dPu, -(w / r) * dPw);
      const float v2 = fmaf(r / nk, V.kpm * dPdr, V.gm * r * r / (d * sqrtf(d)));
      if (v2 > 0.0f) {
        const float g2 = (float)g_v[k] / (2.0f * sqrtf(v2));
        gnk = (double)(-g2 * (r / (nk * nk)) * V.kpm * dPdr);
        const float gd = g2 * (r / nk) * V.kpm;
        axis_d_adjoint(gQ, (long long)j * V.nr, 1, V.nr, i, V.hu, gd * dudr);
        axis_d_adjoint(gQ, i, V.nr, V.nz, j, V.hw, -gd * (w / r));
      }
    }
    g_n[k] = gnk;
  }
}

__global__ void pressure_vphi_adjoint_finish(long long total, const float *__restrict__ n,
                                             const float *__restrict__ T,
                                             const double *__restrict__ gQ, double *g_n,
                                             double *__restrict__ g_T) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    g_n[k] += gQ[k] * (double)__ldg(T + k);
    g_T[k] = gQ[k] * (double)__ldg(n + k);
  }
}

int launch_pressure_vphi_adjoint(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                                 const float *n, const float *T, const double *g_v, double *g_n,
                                 double *g_T, cudaStream_t stream) {
  VphiDev V;
  V.nr = g.nr;
  V.nz = g.nz;
  V.r_log = g.r_log;
  V.r_in = (float)g.r_in_au;
  V.r_out = (float)g.r_out_au;
  V.lnratio = (float)log(g.r_out_au / g.r_in_au);
  V.hu = g.r_log ? (float)(log(g.r_out_au / g.r_in_au) / (g.nr - 1))
                 : (float)((g.r_out_au - g.r_in_au) / (g.nr - 1));
  V.hw = (float)(g.zr_max / (g.nz - 1));
  V.gm = (float)(kChainGMsun * geo.mstar_msun / kChainAu / 1e10);
  V.kpm = (float)(kChainK / (line.m_mol_amu * kChainAmu) / 1e10);
  const long long total = (long long)g.nr * g.nz;
  double *gQ = nullptr;
  cudaError_t e = stream_alloc((void **)&gQ, (size_t)total * sizeof(double), stream);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "rotation adjoint scratch: %s", cudaGetErrorString(e));
  e = cudaMemsetAsync(gQ, 0, (size_t)total * sizeof(double), stream);
  const long long blocks = (total + 255) / 256;
  const unsigned nb = (unsigned)(blocks < 4096 ? blocks : 4096);
  if (e == cudaSuccess) {
    pressure_vphi_adjoint_kernel<<<nb, 256, 0, stream>>>(V, n, T, g_v, g_n, gQ);
    pressure_vphi_adjoint_finish<<<nb, 256, 0, stream>>>(total, n, T, gQ, g_n, g_T);
    e = cudaGetLastError();
  }
  cudaFreeAsync(gQ, stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "rotation adjoint: %s", cudaGetErrorString(e));
  return RT_OK;
}

// Reverse mode of the chain for a scalar loss: dL/dT per node from dL/dn_H2 and dL/d(surfaces),
// one warp per radius column (the forward quantities are recomputed). With
// e_j = exp(-I_j - ln(T_j / T_0)), S = sum_j w_j e_j (trapezoid weights w_j), n_j = Cn e_j,
// Cn = Sigma / (2 S m_mol), and the column N_j = sum_{k >= j} (dz / 2)(n_k + n_{k+1}):
//   h_hi = dw (j* + (N_a - N_d) / (N_a - N_b)) -> dL/dN at the two nodes of its cell;
//   dL/dn_k += (dz / 2)(P_k [k < nz - 1] + P_{k-1} [k > 0]),  P_k = sum_{j <= k} dL/dN_j;
//   dL/de_k = Cn dL/dn_k - (Cn / S) w_k sum_j dL/dn_j e_j;   dL/d ln rho_k = e_k dL/de_k;
//   dL/dI_k = -dL/d ln rho_k;  dL/dT_k += -dL/d ln rho_k / T_k (and the ln T_0 term);
//   I_j = sum_{m=1}^{j} (dz / 2)(g_{m-1} + g_m), g_m = a_m / T_m -> dL/dg_m from suffix sums
//     of dL/dI, dL/dT_m += -dL/dg_m g_m / T_m;
//   h_lo = dw ((j - 1) + (T_f - T_a) / (T_b - T_a)) -> the two nodes of its cell.
// Pass 1 stores e_j in a float scratch column, pass 2 finds the h_hi cell, pass 3 forms
// dL/dn_j (kept in a second scratch column) and sum_j dL/dn_j e_j, pass 4 walks down with the
// suffix sum of dL/dI and writes dL/dT (the FP64 inputs and output are converted once each:
// conversions run on the FP64 pipe).
// FP32 arithmetic (B300's FP64 rate is a small fraction of its FP32 rate; a first FP64 version
// with one thread per column took 3.7 ms on the 512 x 256 grid, the FP32 one 0.22 ms), the
// running sums as warp scans with a carry between 32-node chunks (0.022 ms).
struct ChainAdjDev {
  int nr, nz, r_log;
  float r_in, r_out, zr_max;
  float sigma0, r_c, gamma;
  float A;         // G M m_mol / (k au) [K au]: gravity term per au of height, times 1/T
  float m_mol_g;   // mean molecular mass [g]
  float T_freeze, N_dissoc;
};

// warp scans over the 32 lanes: inclusive prefix (lane l: sum of lanes 0..l) and inclusive
// suffix (lane l: sum of lanes l..31)
__device__ __forceinline__ float warp_prefix(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}
__device__ __forceinline__ float warp_suffix(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += u;
  }
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per radius column: lane l takes nodes 32 c + l of chunk c; the running integrals
// (I upward, the column N and the suffix sum of dL/dI downward) are warp scans with a carry
// between chunks, the crossings come from warp ballots.
__global__ void field_chain_adjoint_kernel(const ChainAdjDev C, const float *__restrict__ T,
                                           const double *__restrict__ g_n,
                                           const double *__restrict__ g_lo,
                                           const double *__restrict__ g_hi, double *g_T,
                                           float *__restrict__ ev, float *__restrict__ gnv) {
  const int nr = C.nr, nz = C.nz;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int nch = (nz + 31) / 32;
  for (long long ii = warp; ii < nr; ii += nwarps) {
    const int i = (int)ii;
    const float t = (float)i / (float)(nr - 1);
    const float r_au = C.r_log ? C.r_in * powf(C.r_out / C.r_in, t) : C.r_in + (C.r_out - C.r_in) * t;
    const float dz_au = C.zr_max / (float)(nz - 1) * r_au;
    const float dz_cm = dz_au * (float)kChainAu;
    auto Tj = [&](int j) { return T[(long long)j * nr + i]; };
    auto grav = [&](int j) {
      const float z = dz_au * (float)j, d2 = r_au * r_au + z * z;
      return C.A * z / (d2 * sqrtf(d2)) / Tj(j);
    };
    auto at = [&](int j) { return (long long)j * nr + i; };
    const float T0 = Tj(0);
    // pass 1 (upward): e_j and S / dz
    float carryI = 0.0f, gprev = 0.0f, eprev = 0.0f, Ssum = 0.0f;
    for (int c = 0; c < nch; c++) {
      const int j = 32 * c + lane;
      const bool in = j < nz;
      const float g = in ? grav(j) : 0.0f;
      float gl = __shfl_up_sync(0xffffffffu, g, 1);
      if (lane == 0) gl = gprev;
      const float term = (in && j >= 1) ? 0.5f * dz_au * (gl + g) : 0.0f;
      const float I = carryI + warp_prefix(term, lane);
      const float e = in ? expf(-I - logf(Tj(j) / T0)) : 0.0f;
      if (in) ev[at(j)] = e;
      float el = __shfl_up_sync(0xffffffffu, e, 1);
      if (lane == 0) el = eprev;
      Ssum += warp_sum((in && j >= 1) ? 0.5f * (el + e) : 0.0f);
      carryI = __shfl_sync(0xffffffffu, I, 31);
      gprev = __shfl_sync(0xffffffffu, g, 31);
      eprev = __shfl_sync(0xffffffffu, e, 31);
    }
    const float x = r_au / C.r_c;
    const float sigma = C.sigma0 * powf(x, -C.gamma) * expf(-powf(x, 2.0f - C.gamma));
    const float Sdz = Ssum;
    const float Cn = sigma / (2.0f * Sdz * dz_cm) / C.m_mol_g;
    const float dw = C.zr_max / (float)(nz - 1);
    __syncwarp();
    // pass 2 (downward): the h_hi cell and dL/dN at its two nodes
    int js = nz;
    float gNa = 0.0f, gNb = 0.0f;
    const float ghi = g_hi ? (float)g_hi[i] : 0.0f;
    if (ghi != 0.0f) {
      float carryN = 0.0f, eabove = 0.0f;
      for (int c = nch - 1; c >= 0; c--) {
        const int j = 32 * c + lane;
        const bool in = j < nz;
        const float e = in ? ev[at(j)] : 0.0f;
        float eu = __shfl_down_sync(0xffffffffu, e, 1);
        if (lane == 31) eu = eabove;
        const float u = (in && j <= nz - 2) ? 0.5f * dz_cm * Cn * (e + eu) : 0.0f;
        const float N = carryN + warp_suffix(u, lane);
        const unsigned hit = __ballot_sync(0xffffffffu, in && 0.706f * N > C.N_dissoc);
        if (hit) {
          const int lh = 31 - __clz(hit);  // highest node of the chunk over the threshold
          const float Nj = __shfl_sync(0xffffffffu, N, lh);
          const float uj = __shfl_sync(0xffffffffu, u, lh);
          const float Na = 0.706f * Nj, Nb = 0.706f * (Nj - uj), dN = Na - Nb;
          gNa = ghi * dw * ((C.N_dissoc - Nb) / dN) / dN * 0.706f;
          gNb = ghi * dw * ((Na - C.N_dissoc) / dN) / dN * 0.706f;
          js = 32 * c + lh;
          break;
        }
        carryN = __shfl_sync(0xffffffffu, N, 0);
        eabove = __shfl_sync(0xffffffffu, e, 0);
      }
    }
    // pass 3: dL/dn_j (scratch) and sum_j dL/dn_j e_j
    float dot = 0.0f;
    for (int c = 0; c < nch; c++) {
      const int j = 32 * c + lane;
      if (j < nz) {
        float v = g_n ? (float)g_n[at(j)] : 0.0f;
        const float Pk = (j >= js ? gNa : 0.0f) + (j >= js + 1 ? gNb : 0.0f);
        const float Pk1 = (j - 1 >= js ? gNa : 0.0f) + (j >= js + 2 ? gNb : 0.0f);
        if (j <= nz - 2) v += 0.5f * dz_cm * Pk;
        if (j >= 1) v += 0.5f * dz_cm * Pk1;
        gnv[at(j)] = v;
        dot += v * ev[at(j)];
      }
    }
    const float ge_dot = warp_sum(dot);
    // pass 4 (downward): Q_m = sum_{j > m} dL/dI_j, dL/dT
    float carryQ = 0.0f, sglr = 0.0f;
    for (int c = nch - 1; c >= 0; c--) {
      const int m = 32 * c + lane;
      const bool in = m < nz;
      float glr = 0.0f;
      if (in) {
        const float wk = (m > 0 ? 0.5f : 0.0f) + (m < nz - 1 ? 0.5f : 0.0f);
        glr = (Cn * gnv[at(m)] - Cn / Sdz * wk * ge_dot) * ev[at(m)];
      }
      const float gI = -glr;
      const float incl = carryQ + warp_suffix(gI, lane);
      const float Q = incl - gI;  // exclusive: nodes above m
      if (in) {
        float gg = 0.0f;
        if (m + 1 <= nz - 1) gg += 0.5f * dz_au * Q;
        if (m >= 1) gg += 0.5f * dz_au * (Q + gI);
        g_T[at(m)] = (double)(-glr / Tj(m) - gg * grav(m) / Tj(m));
      }
      sglr += glr;
      carryQ = __shfl_sync(0xffffffffu, incl, 0);
    }
    sglr = warp_sum(sglr);
    __syncwarp();
    if (lane == 0) g_T[at(0)] += (double)(sglr / T0);  // the ln T_0 term (zero up to rounding)
    // h_lo: lowest cell [j-1, j] with T_j > T_freeze (none when the midplane node is warmer)
    const float glo = g_lo ? (float)g_lo[i] : 0.0f;
    if (glo != 0.0f && !(T0 > C.T_freeze)) {
      for (int c = 0; c < nch; c++) {
        const int j = 32 * c + lane;
        const unsigned hit = __ballot_sync(0xffffffffu, j >= 1 && j < nz && Tj(j) > C.T_freeze);
        if (hit) {
          const int jl = 32 * c + __ffs(hit) - 1;
          __syncwarp();
          if (lane == 0) {
            const float Ta = Tj(jl - 1), Tb = Tj(jl), q = (Tb - Ta) * (Tb - Ta);
            g_T[at(jl - 1)] += (double)(glo * dw * (C.T_freeze - Tb) / q);
            g_T[at(jl)] += (double)(-glo * dw * (C.T_freeze - Ta) / q);
          }
          break;
        }
      }
    }
    __syncwarp();
  }
}

int launch_field_chain_adjoint(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                               const rt_chain &c, const float *T, const double *g_n,
                               const double *g_lo, const double *g_hi, double *g_T,
                               cudaStream_t stream) {
  ChainAdjDev C;
  C.nr = g.nr;
  C.nz = g.nz;
  C.r_log = g.r_log;
  C.r_in = (float)g.r_in_au;
  C.r_out = (float)g.r_out_au;
  C.zr_max = (float)g.zr_max;
  C.sigma0 = (float)c.sigma0_gcm2;
  C.r_c = (float)c.r_c_au;
  C.gamma = (float)c.gamma;
  const double m = line.m_mol_amu * kChainAmu;
  C.A = (float)(kChainGMsun * geo.mstar_msun * m / (kChainK * kChainAu));
  C.m_mol_g = (float)m;
  C.T_freeze = (float)c.T_freeze_K;
  C.N_dissoc = (float)c.N_dissoc_cm2;
  const size_t col = (size_t)g.nr * g.nz;
  float *scr = nullptr;
  cudaError_t e = stream_alloc((void **)&scr, 2 * col * sizeof(float), stream);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "chain adjoint scratch: %s", cudaGetErrorString(e));
  const int threads = 128;  // four columns (warps) per block
  const long long blocks = ((long long)g.nr * 32 + threads - 1) / threads;
  field_chain_adjoint_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, g_n, g_lo, g_hi, g_T,
                                                                       scr, scr + col);
  e = cudaGetLastError();
  cudaFreeAsync(scr, stream);
  if (e != cudaSuccess)
    return set_error(RT_ECUDA, "field chain adjoint launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

int launch_field_chain(const rt_grid &g, const rt_geom &geo, const rt_line &line,
                       const rt_chain &c, const float *T, float *n, float *N, float *h_lo,
                       float *h_hi, cudaStream_t stream) {
  ChainDev C;
  C.nr = g.nr;
  C.nz = g.nz;
  C.r_log = g.r_log;
  C.r_in = (float)g.r_in_au;
  C.r_out = (float)g.r_out_au;
  C.zr_max = g.zr_max;
  C.sigma0 = (float)c.sigma0_gcm2;
  C.r_c = (float)c.r_c_au;
  C.gamma = (float)c.gamma;
  const double m = line.m_mol_amu * kChainAmu;
  C.A = (float)(kChainGMsun * geo.mstar_msun * m / (kChainK * kChainAu));
  C.m_mol_g = (float)m;
  C.T_freeze = (float)c.T_freeze_K;
  C.N_dissoc = (float)c.N_dissoc_cm2;
  const int threads = 256;  // 8 columns per block
  const long long blocks = ((long long)g.nr * 32 + threads - 1) / threads;
  field_chain_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, n, N, h_lo, h_hi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "field chain launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rtb
