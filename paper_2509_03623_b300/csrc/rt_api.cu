// C-ABI entry points, argument validation, error reporting and the host-side construction
// of the per-launch parameter block (unit conversions, molecular constants, LTE table).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "rt_internal.cuh"

namespace rtb {

// CGS constants (CODATA 2018 exact SI-defining values; IAU 2012/2015 nominal values).
static const double kH = 6.62607015e-27;       // erg s
static const double kK = 1.380649e-16;         // erg / K
static const double kC = 2.99792458e10;        // cm / s
static const double kAmu = 1.66053906660e-24;  // g
static const double kGMsun = 1.3271244e26;     // cm^3 s^-2
static const double kAu = 1.495978707e13;      // cm
static const double kPi = 3.14159265358979323846;
static const double kLog2e = 1.4426950408889634;

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = 0; }

static bool is_finite(double x) { return isfinite(x) != 0; }

// Rigid-rotor level statistics at temperature T: lower-level fraction
// f_l = g_l exp(-E_l/kT)/Z and mean level energy <E>.
static void rotor_stats(double T, double B, int Jl, double *fl, double *meanE) {
  double Z = 0.0, EZ = 0.0;
  for (int J = 0; J < 200000; J++) {
    double E = kH * B * J * (J + 1.0);
    double w = (2.0 * J + 1.0) * exp(-E / (kK * T));
    Z += w;
    EZ += E * w;
    if (J > Jl + 2 && w < 1e-18 * Z) break;
  }
  double El = kH * B * Jl * (Jl + 1.0);
  *fl = (2.0 * Jl + 1.0) * exp(-El / (kK * T)) / Z;
  *meanE = EZ / Z;
}

// LTE opacity factor F(T) = f_l(T) (1 - exp(-dE/kT)) as Phi = log2 F on t = log2 T, with
// dPhi/dt = d ln F / d ln T = (E_l - <E>)/kT - x e^-x / (1 - e^-x), x = dE/kT; cubic Hermite
// segments in Horner form.
static void build_table(double B, int Ju, float *tab) {
  int Jl = Ju - 1;
  double El = kH * B * Jl * (Jl + 1.0);
  double dE = kH * B * (Ju * (Ju + 1.0) - Jl * (Jl + 1.0));
  double y[kTabN], m[kTabN];
  const double h = 1.0 / kTabInvH;
  for (int i = 0; i < kTabN; i++) {
    double T = exp2(kTabT0 + i * h);
    double fl, mE;
    rotor_stats(T, B, Jl, &fl, &mE);
    double x = dE / (kK * T);
    double one_m = -expm1(-x);
    y[i] = log2(fl * one_m);
    m[i] = ((El - mE) / (kK * T) - x * exp(-x) / one_m) * h;
  }
  for (int i = 0; i < kTabSeg; i++) {
    double y0 = y[i], y1 = y[i + 1], m0 = m[i], m1 = m[i + 1];
    tab[4 * i + 0] = (float)y0;
    tab[4 * i + 1] = (float)m0;
    tab[4 * i + 2] = (float)(3.0 * (y1 - y0) - 2.0 * m0 - m1);
    tab[4 * i + 3] = (float)(2.0 * (y0 - y1) + m0 + m1);
  }
}

// The table depends only on (B, J_u); the last few are cached so that repeated renders of
// the same line do not recompute ~10^5 exponentials on the host.
static void lte_table(double B, int Ju, float *tab) {
  struct Entry {
    double B;
    int Ju;
    float tab[kTabSeg * 4];
  };
  static std::mutex mu;
  static Entry cache[4];
  static int n_cached = 0, next = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n_cached; i++)
      if (cache[i].B == B && cache[i].Ju == Ju) {
        memcpy(tab, cache[i].tab, sizeof(cache[i].tab));
        return;
      }
  }
  build_table(B, Ju, tab);
  std::lock_guard<std::mutex> lk(mu);
  Entry &e = cache[next];
  e.B = B;
  e.Ju = Ju;
  memcpy(e.tab, tab, sizeof(e.tab));
  next = (next + 1) % 4;
  if (n_cached < 4) n_cached++;
}

cudaError_t stream_alloc(void **p, size_t bytes, cudaStream_t stream) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props;
      memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pools[dev], &props);
      if (e != cudaSuccess) {
        pools[dev] = nullptr;
        return e;
      }
      unsigned long long keep = kPoolKeepBytes;
      cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, stream);
}

// Validation of the geometry, view and line shared by every render entry point.
static int check_common(const rt_geom &o, const rt_view &v, const rt_line &l) {
  if (!is_finite(o.incl_deg) || !is_finite(o.pa_deg) || !is_finite(o.mstar_msun) || o.mstar_msun < 0 ||
      !is_finite(o.vsys_kms))
    return set_error(RT_EINVAL, "geometry must be finite with mstar >= 0");
  if (v.nx < 0 || v.ny < 0) return set_error(RT_EINVAL, "negative image size");
  // (the kernels' 32-bit work counters count at most this many rays, plus one per warp)
  if ((long long)v.nx * v.ny > (1LL << 31)) return set_error(RT_EINVAL, "more than 2^31 pixels");
  if (v.nch < 0 || v.nch > RT_MAX_CH)
    return set_error(RT_EINVAL, "nch must be in [0, %d] (got %d)", RT_MAX_CH, v.nch);
  if (v.nch > 0 && !v.v_kms) return set_error(RT_EINVAL, "null channel velocities");
  if (v.n_samples < 1 || v.n_samples > (1 << 20))
    return set_error(RT_EINVAL, "n_samples must be in [1, 2^20]");
  if (!is_finite(v.I0) || !is_finite(v.half_fov_au)) return set_error(RT_EINVAL, "non-finite view");
  if (v.units != 0 && v.units != 1) return set_error(RT_EINVAL, "units must be 0 or 1");
  if (v.units == 1 && !(is_finite(o.dist_pc) && o.dist_pc > 0))
    return set_error(RT_EINVAL, "dist_pc must be > 0 for Jy per pixel");
  if (!(is_finite(l.nu0_hz) && l.nu0_hz > 0) || !(is_finite(l.A_ul) && l.A_ul >= 0) || l.J_u < 1 ||
      !(is_finite(l.m_co_amu) && l.m_co_amu > 0) || !(is_finite(l.m_mol_amu) && l.m_mol_amu > 0) ||
      !is_finite(l.B_rot_hz))
    return set_error(RT_EINVAL, "invalid line constants");
  for (int c = 0; c < v.nch; c++)
    if (!is_finite(v.v_kms[c])) return set_error(RT_EINVAL, "non-finite channel velocity %d", c);

  return RT_OK;
}

// Parameters shared by every render (geometry, image, channels, line, LTE table); r_fov: the
// extent whose 1.1 times sets the default half field of view.
static void fill_common(const rt_geom &o, const rt_view &v, const rt_line &l, double r_fov,
                        MarchParams *P) {
  P->c_th = (float)(2.0 * kK / (l.m_co_amu * kAmu) / 1e10);
  P->c_mach = (float)(2.0 * kK / (l.m_mol_amu * kAmu) / 1e10);

  double inc = o.incl_deg * kPi / 180.0, pa = o.pa_deg * kPi / 180.0;
  P->sin_i = sin(inc);
  P->sin_if = (float)P->sin_i;
  P->cos_i = cos(inc);
  P->sin_pa = sin(pa);
  P->cos_pa = cos(pa);
  // reciprocals for the per-ray setup (the device then multiplies instead of dividing: FP64
  // division is a long instruction sequence on this part's narrow FP64 pipe)
  P->inv_wy = P->sin_i != 0.0 ? 1.0 / P->sin_i : 0.0;
  P->inv_wz = P->cos_i != 0.0 ? -1.0 / P->cos_i : 0.0;
  P->inv_2a = P->sin_i != 0.0 ? 0.5 / (P->sin_i * P->sin_i) : 0.0;
  P->inv_ns = v.n_samples > 0 ? 1.0 / v.n_samples : 0.0;
  double hf = v.half_fov_au > 0 ? v.half_fov_au : 1.1 * r_fov;
  P->px = v.nx > 0 ? 2.0 * hf / v.nx : 0.0;
  P->py = v.ny > 0 ? 2.0 * hf / v.ny : 0.0;
  P->vk = (float)(sqrt(kGMsun * o.mstar_msun / kAu) / 1e5);
  P->vsys = (float)o.vsys_kms;

  P->nx = v.nx;
  P->ny = v.ny;
  P->nch = v.nch;
  P->n_samples = v.n_samples;
  int kb = 0;
  while ((1LL << kb) < (long long)v.n_samples) kb++;  // bits of the largest sample index
  P->step_bits = 24 - kb;
  // double-float copies for the FP32 ray setup of the disk (pixel centres (i + 1/2 - n/2)
  // are exact in FP32 below 2^22 pixels a side)
  auto f2 = [](double d) {
    F2 r;
    r.hi = (float)d;
    r.lo = (float)(d - (double)r.hi);
    return r;
  };
  P->f_px = f2(P->px);
  P->f_py = f2(P->py);
  P->f_cos_pa = f2(P->cos_pa);
  P->f_sin_pa = f2(P->sin_pa);
  P->f_cos_i = f2(P->cos_i);
  P->f_sin_i = f2(P->sin_i);
  P->f_H = f2(P->H_cyl);
  P->f_R = f2(P->R_cyl);
  P->f_R2 = f2(P->R_cyl * P->R_cyl);
  P->f_4a = f2(4.0 * P->sin_i * P->sin_i);
  P->f_inv_wz = f2(P->inv_wz);
  P->f_inv_2a = f2(P->inv_2a);
  P->f_inv_ns = f2(P->inv_ns);
  P->f_vks = f2((double)P->vk * P->sin_i);
  P->f2_setup = (!P->box && !P->sph && v.nx <= (1 << 22) && v.ny <= (1 << 22)) ? 1 : 0;
  double B_nu = 2.0 * kH * pow(l.nu0_hz, 3) / (kC * kC);  // 2 h nu0^3 / c^2
  double conv = 1.0;
  if (v.units == 1) {
    double arcsec = kPi / 648000.0;
    conv = (P->px / o.dist_pc * arcsec) * (P->py / o.dist_pc * arcsec) * 1e23;
  }
  P->out_scale = (float)(B_nu * conv);
  P->I0 = (float)v.I0;

  double B = l.B_rot_hz > 0 ? l.B_rot_hz : l.nu0_hz / (2.0 * l.J_u);
  int Ju = l.J_u, Jl = l.J_u - 1;
  double dE = kH * B * (Ju * (Ju + 1.0) - Jl * (Jl + 1.0));
  // B_ul = A c^2 / (2 h nu0^3), B_lu = (g_u/g_l) B_ul; optical depth per
  // (n_CO F inv_alpha[s/km] ds[au]) = (h nu0 / 4 pi) B_lu c / (nu0 sqrt(pi)) / 1e5 * au
  double Bul = l.A_ul * kC * kC / (2.0 * kH * pow(l.nu0_hz, 3));
  double Blu = (2.0 * Ju + 1.0) / (2.0 * Jl + 1.0) * Bul;
  double kap = kH * l.nu0_hz / (4.0 * kPi) * Blu * kC / (l.nu0_hz * sqrt(kPi)) / 1e5 * kAu;
  P->kappa_k = (float)(kap * kLog2e);
  P->theta_s = (float)(dE / kK * kLog2e);
  for (int c = 0; c < v.nch; c++) P->v[c] = v.v_kms[c];
  // Equal spacing (to float rounding) lets the kernels form v_c = v0 + c dv in registers.
  P->v_uniform = 0;
  if (v.nch >= 2) {
    double v0 = v.v_kms[0], dv = ((double)v.v_kms[v.nch - 1] - v0) / (v.nch - 1);
    bool uni = dv != 0.0;
    for (int c = 0; c < v.nch && uni; c++) {
      double e = fabs((double)v.v_kms[c] - (v0 + c * dv));
      if (e > 4e-7 * (fabs(v0) + fabs(dv) * v.nch)) uni = false;
    }
    if (uni) {
      P->v_uniform = 1;
      P->v0 = (float)v0;
      P->dv = (float)dv;
    }
  }
  lte_table(B, Ju, P->tab);
}

int build_params(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                 const rt_view *view, const rt_line *line, MarchParams *P) {
  if (!grid || !fields || !geom || !view || !line || !P)
    return set_error(RT_EINVAL, "null argument struct");
  const rt_grid &g = *grid;
  const rt_fields &f = *fields;
  const rt_geom &o = *geom;
  const rt_view &v = *view;
  const rt_line &l = *line;
  if (g.nr < 2 || g.nz < 2 || (long long)g.nr * g.nz > (1LL << 28))
    return set_error(RT_EINVAL, "grid needs 2 <= nr, nz and nr*nz <= 2^28 (got %d x %d)", g.nr,
                     g.nz);
  if (!is_finite(g.r_in_au) || !is_finite(g.r_out_au) || !(g.r_in_au > 0) ||
      !(g.r_out_au > g.r_in_au))
    return set_error(RT_EINVAL, "grid radii need 0 < r_in < r_out");
  if (!is_finite(g.zr_max) || !(g.zr_max > 0)) return set_error(RT_EINVAL, "zr_max must be > 0");
  if (!f.T_K || !f.n_h2_cm3 || !f.vturb || !f.h_lo || !f.h_hi)
    return set_error(RT_EINVAL, "null field pointer");
  if (!is_finite(f.x_co) || f.x_co < 0) return set_error(RT_EINVAL, "x_co must be finite and >= 0");
  if (!is_finite(f.edge_w) || f.edge_w < 0) return set_error(RT_EINVAL, "edge_w must be >= 0");
  int rc = check_common(o, v, l);
  if (rc != RT_OK) return rc;

  memset(P, 0, sizeof(*P));
  P->nr = g.nr;
  P->nz = g.nz;
  P->r_log = g.r_log ? 1 : 0;
  if (P->r_log) {
    P->lr_scale = (float)(0.5 * (g.nr - 1) / log2(g.r_out_au / g.r_in_au));
    P->lr_off = 0.0f;
  } else {
    double s = (g.nr - 1) / (g.r_out_au - g.r_in_au);
    P->lr_scale = (float)s;
    P->lr_off = (float)(-g.r_in_au * s);
  }
  P->r_in2 = (float)(g.r_in_au * g.r_in_au);
  P->inv_rin2 = (float)(1.0 / (g.r_in_au * g.r_in_au));
  P->zr_max = (float)g.zr_max;
  P->zr_max2 = (float)(g.zr_max * g.zr_max);
  P->w_scale = (float)((g.nz - 1) / g.zr_max);
  P->T = f.T_K;
  P->n = f.n_h2_cm3;
  P->vt = f.vturb;
  P->hlo = f.h_lo;
  P->hhi = f.h_hi;
  P->vphi = f.vphi_kms;
  P->x_co = (float)f.x_co;
  P->hard_edge = f.edge_w > 0 ? 0 : 1;
  P->edge_k = f.edge_w > 0 ? (float)(kLog2e / f.edge_w) : 0.0f;
  P->vturb_mach = f.vturb_mach ? 1 : 0;
  P->R_cyl = g.r_out_au;
  P->H_cyl = g.zr_max * g.r_out_au;
  fill_common(o, v, l, g.r_out_au, P);
  return RT_OK;
}

// Node records of a 3-D grid: {T, n_H2, v_turb, x_co} and {vx, vy, vz, 0} per node.
__global__ void pack_nodes3_kernel(const rt_fields3 f, long long n, float4 *__restrict__ a,
                                   float4 *__restrict__ b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    a[i] = make_float4(f.T_K[i], f.n_h2_cm3[i], f.vturb[i], f.x_co[i]);
    b[i] = make_float4(f.vx_kms[i], f.vy_kms[i], f.vz_kms[i], 0.0f);
  }
}

// The parameters of a 3-D Cartesian render from the grid and the turbulence mode (the field
// pointers are checked by the callers that read them).
static int build_params3_core(const rt_grid3 *grid, int vturb_mach, const rt_geom *geom,
                              const rt_view *view, const rt_line *line, MarchParams *P);

static int build_params3(const rt_grid3 *grid, const rt_fields3 *fields, const rt_geom *geom,
                         const rt_view *view, const rt_line *line, MarchParams *P) {
  if (!fields) return set_error(RT_EINVAL, "null argument struct");
  const rt_fields3 &f = *fields;
  if (!f.T_K || !f.n_h2_cm3 || !f.vturb || !f.x_co || !f.vx_kms || !f.vy_kms || !f.vz_kms)
    return set_error(RT_EINVAL, "null field pointer");
  return build_params3_core(grid, f.vturb_mach, geom, view, line, P);
}

static int build_params3_core(const rt_grid3 *grid, int vturb_mach, const rt_geom *geom,
                              const rt_view *view, const rt_line *line, MarchParams *P) {
  if (!grid || !geom || !view || !line || !P)
    return set_error(RT_EINVAL, "null argument struct");
  const rt_grid3 &g = *grid;
  if (g.nx < 2 || g.ny < 2 || g.nz < 2 || (long long)g.nx * g.ny * g.nz > (1LL << 28))
    return set_error(RT_EINVAL, "3-D grid needs >= 2 nodes per axis and <= 2^28 nodes "
                     "(got %d x %d x %d)", g.nx, g.ny, g.nz);
  const double ext[6] = {g.x0_au, g.x1_au, g.y0_au, g.y1_au, g.z0_au, g.z1_au};
  for (int k = 0; k < 6; k++)
    if (!is_finite(ext[k])) return set_error(RT_EINVAL, "non-finite box extent");
  if (!(g.x1_au > g.x0_au) || !(g.y1_au > g.y0_au) || !(g.z1_au > g.z0_au))
    return set_error(RT_EINVAL, "box extents need x0 < x1, y0 < y1, z0 < z1");
  int rc = check_common(*geom, *view, *line);
  if (rc != RT_OK) return rc;
  memset(P, 0, sizeof(*P));
  P->box = 1;
  P->bx0 = g.x0_au;
  P->bx1 = g.x1_au;
  P->by0 = g.y0_au;
  P->by1 = g.y1_au;
  P->bz0 = g.z0_au;
  P->bz1 = g.z1_au;
  P->n3x = g.nx;
  P->n3y = g.ny;
  P->n3z = g.nz;
  // per axis the node nearest the middle of the box, its position and the nodes per au
  auto axis = [](double a0, double a1, int n, int *k, float *c, float *s) {
    const double sc = (n - 1) / (a1 - a0);
    int kk = (int)floor(-a0 * sc + 0.5);  // node nearest coordinate 0 ...
    kk = kk < 0 ? 0 : (kk > n - 1 ? n - 1 : kk);  // ... inside the grid
    *k = kk;
    *c = (float)(a0 + kk / sc);
    *s = (float)sc;
  };
  axis(g.x0_au, g.x1_au, g.nx, &P->g3kx, &P->g3cx, &P->g3sx);
  axis(g.y0_au, g.y1_au, g.ny, &P->g3ky, &P->g3cy, &P->g3sy);
  axis(g.z0_au, g.z1_au, g.nz, &P->g3kz, &P->g3cz, &P->g3sz);
  P->vturb_mach = vturb_mach ? 1 : 0;
  double reach = 0.0;
  for (int k = 0; k < 6; k++) reach = fmax(reach, fabs(ext[k]));
  fill_common(*geom, *view, *line, reach, P);
  P->cos_if = (float)P->cos_i;
  return RT_OK;
}

// The parameters of a spherical render from the grid and the turbulence mode (the field
// pointers are checked by the callers that read them).
static int build_params_sph_core(const rt_grid_sph *grid, int vturb_mach, const rt_geom *geom,
                                 const rt_view *view, const rt_line *line, MarchParams *P);

static int build_params_sph(const rt_grid_sph *grid, const rt_fields_sph *fields,
                            const rt_geom *geom, const rt_view *view, const rt_line *line,
                            MarchParams *P) {
  if (!fields) return set_error(RT_EINVAL, "null argument struct");
  const rt_fields_sph &f = *fields;
  if (!f.T_K || !f.n_h2_cm3 || !f.vturb || !f.x_co || !f.vr_kms || !f.vth_kms || !f.vph_kms)
    return set_error(RT_EINVAL, "null field pointer");
  return build_params_sph_core(grid, f.vturb_mach, geom, view, line, P);
}

static int build_params_sph_core(const rt_grid_sph *grid, int vturb_mach, const rt_geom *geom,
                                 const rt_view *view, const rt_line *line, MarchParams *P) {
  if (!grid || !geom || !view || !line || !P)
    return set_error(RT_EINVAL, "null argument struct");
  const rt_grid_sph &g = *grid;
  if (g.nr < 2 || g.nth < 2 || g.nph < 1 || (long long)g.nr * g.nth * g.nph > (1LL << 28))
    return set_error(RT_EINVAL, "spherical grid needs nr, nth >= 2, nph >= 1 and <= 2^28 "
                     "nodes (got %d x %d x %d)", g.nr, g.nth, g.nph);
  if (!is_finite(g.r_in_au) || !is_finite(g.r_out_au) || !(g.r_in_au >= 0) ||
      !(g.r_out_au > g.r_in_au) || (g.r_log && !(g.r_in_au > 0)))
    return set_error(RT_EINVAL, "spherical grid radii need 0 <= r_in < r_out (0 < r_in on a "
                     "log grid)");
  if (!is_finite(g.th0_rad) || !is_finite(g.th1_rad) || !(g.th0_rad >= 0) ||
      !(g.th1_rad > g.th0_rad) || !(g.th1_rad <= 3.14159265358979323846))
    return set_error(RT_EINVAL, "colatitudes need 0 <= th0 < th1 <= pi");
  int rc = check_common(*geom, *view, *line);
  if (rc != RT_OK) return rc;
  memset(P, 0, sizeof(*P));
  P->sph = 1;
  P->snr = g.nr;
  P->snth = g.nth;
  P->snph = g.nph;
  P->r_log = g.r_log ? 1 : 0;
  if (P->r_log) {
    P->lr_scale = (float)(0.5 * (g.nr - 1) / log2(g.r_out_au / g.r_in_au));
    P->lr_off = 0.0f;
    P->inv_rin2 = (float)(1.0 / (g.r_in_au * g.r_in_au));
  } else {
    const double sc = (g.nr - 1) / (g.r_out_au - g.r_in_au);
    P->lr_scale = (float)sc;
    P->lr_off = (float)(-g.r_in_au * sc);
  }
  P->r_in2 = (float)(g.r_in_au * g.r_in_au);
  P->r_out2 = (float)(g.r_out_au * g.r_out_au);
  P->th0 = (float)g.th0_rad;
  P->th1 = (float)g.th1_rad;
  P->th_scale = (float)((g.nth - 1) / (g.th1_rad - g.th0_rad));
  P->ph_scale = (float)(g.nph / (2.0 * 3.14159265358979323846));
  P->R_cyl = g.r_out_au;
  P->vturb_mach = vturb_mach ? 1 : 0;
  fill_common(*geom, *view, *line, g.r_out_au, P);
  P->cos_if = (float)P->cos_i;
  return RT_OK;
}

// Node records {T, n, vt, x_co} and three velocity components per node, for the packing
// kernel (the Cartesian and spherical grids share it).
static int pack_and_march(const MarchParams &P0, const rt_fields3 &f, long long nodes,
                          float *cube, cudaStream_t st) {
  float4 *buf = nullptr;
  cudaError_t e = stream_alloc((void **)&buf, (size_t)nodes * 2 * sizeof(float4), st);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "node records (%lld nodes): %s", nodes, cudaGetErrorString(e));
  int rc = RT_OK;
  const long long nb = (nodes + 255) / 256;
  pack_nodes3_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(f, nodes, buf,
                                                                     buf + nodes);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    rc = set_error(RT_ECUDA, "node packing: %s", cudaGetErrorString(e));
  } else {
    MarchParams *P = new (std::nothrow) MarchParams(P0);
    if (!P) {
      rc = set_error(RT_ENOMEM, "host allocation failed");
    } else {
      P->node_a = buf;
      P->node_b = buf + nodes;
      rc = launch_forward(*P, cube, st);
      delete P;
    }
  }
  cudaFreeAsync(buf, st);
  return rc;
}

}  // namespace rtb

using namespace rtb;

extern "C" int rt_render_sph(const rt_grid_sph *grid, const rt_fields_sph *fields,
                             const rt_geom *geom, const rt_view *view, const rt_line *line,
                             float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params_sph(grid, fields, geom, view, line, P);
  const long long npix = rc == RT_OK ? (long long)P->nx * P->ny : 0;
  if (rc == RT_OK && npix * P->nch > 0 && !cube) rc = set_error(RT_EINVAL, "null cube pointer");
  if (rc == RT_OK && npix * P->nch > 0) {
    rt_fields3 f3;
    f3.T_K = fields->T_K;
    f3.n_h2_cm3 = fields->n_h2_cm3;
    f3.vturb = fields->vturb;
    f3.x_co = fields->x_co;
    f3.vx_kms = fields->vr_kms;
    f3.vy_kms = fields->vth_kms;
    f3.vz_kms = fields->vph_kms;
    f3.vturb_mach = fields->vturb_mach;
    rc = pack_and_march(*P, f3, (long long)grid->nr * grid->nth * grid->nph, cube,
                        (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render3d(const rt_grid3 *grid3, const rt_fields3 *fields3,
                           const rt_geom *geom, const rt_view *view, const rt_line *line,
                           float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params3(grid3, fields3, geom, view, line, P);
  const long long npix = rc == RT_OK ? (long long)P->nx * P->ny : 0;
  if (rc == RT_OK && npix * P->nch > 0 && !cube) rc = set_error(RT_EINVAL, "null cube pointer");
  if (rc == RT_OK && npix * P->nch > 0)
    rc = pack_and_march(*P, *fields3, (long long)grid3->nx * grid3->ny * grid3->nz, cube,
                        (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

namespace rtb {

// Argument checks, node packing and the fused adjoint on a 3-D grid (P built by
// build_params3(_core) or build_params_sph(_core)): from the fields f3 (in the packing order),
// packed here, or from records already packed by rt_pack_nodes3 (f3 then unused).
static int adjoint3_call(MarchParams &P, const rt_fields3 *f3, const void *packed,
                         long long nodes, const float *dL_dcube, const float *target,
                         float *cube_out, const rt_grads3 *grads, cudaStream_t st) {
  if (!grads || !grads->dT || !grads->dn_h2 || !grads->dvturb || !grads->dx_co || !grads->dvx ||
      !grads->dvy || !grads->dvz)
    return set_error(RT_EINVAL, "null gradient output");
  const long long n = (long long)P.nx * P.ny * P.nch;
  if (n > 0 && ((dL_dcube == nullptr) == (target == nullptr)))
    return set_error(RT_EINVAL, "give exactly one of dL_dcube and target");
  if (n == 0) {  // no ray or no channel: the gradients are zero
    cudaError_t e = cudaSuccess;
    double *out[7] = {grads->dT, grads->dn_h2, grads->dvturb, grads->dx_co,
                      grads->dvx, grads->dvy, grads->dvz};
    for (int k = 0; k < 7 && e == cudaSuccess; k++)
      e = cudaMemsetAsync(out[k], 0, (size_t)nodes * sizeof(double), st);
    if (e == cudaSuccess && grads->loss) e = cudaMemsetAsync(grads->loss, 0, sizeof(double), st);
    if (e != cudaSuccess) return set_error(RT_ECUDA, "memset: %s", cudaGetErrorString(e));
    return RT_OK;
  }
  if (packed) {  // node records packed by rt_pack_nodes3
    if (reinterpret_cast<uintptr_t>(packed) & 15)
      return set_error(RT_EINVAL, "records must be a 16-byte aligned device pointer");
    P.node_a = static_cast<const float4 *>(packed);
    P.node_b = P.node_a + nodes;
    return launch_adjoint3(P, dL_dcube, target, cube_out, *grads, st);
  }
  float4 *buf = nullptr;
  cudaError_t e = stream_alloc((void **)&buf, (size_t)nodes * 2 * sizeof(float4), st);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "node records (%lld nodes): %s", nodes, cudaGetErrorString(e));
  int rc = RT_OK;
  const long long nb = (nodes + 255) / 256;
  pack_nodes3_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(*f3, nodes, buf,
                                                                        buf + nodes);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    rc = set_error(RT_ECUDA, "node packing: %s", cudaGetErrorString(e));
  } else {
    P.node_a = buf;
    P.node_b = buf + nodes;
    rc = launch_adjoint3(P, dL_dcube, target, cube_out, *grads, st);
  }
  cudaFreeAsync(buf, st);
  return rc;
}

}  // namespace rtb

extern "C" int rt_render3d_adjoint(const rt_grid3 *grid3, const rt_fields3 *fields3,
                                   const rt_geom *geom, const rt_view *view,
                                   const rt_line *line, const float *dL_dcube,
                                   const float *target, float *cube_out,
                                   const rt_grads3 *grads, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params3(grid3, fields3, geom, view, line, P);
  if (rc == RT_OK)
    rc = adjoint3_call(*P, fields3, nullptr, (long long)grid3->nx * grid3->ny * grid3->nz,
                       dL_dcube, target, cube_out, grads, (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_sph_adjoint(const rt_grid_sph *grid, const rt_fields_sph *fields,
                                     const rt_geom *geom, const rt_view *view,
                                     const rt_line *line, const float *dL_dcube,
                                     const float *target, float *cube_out,
                                     const rt_grads3 *grads, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params_sph(grid, fields, geom, view, line, P);
  if (rc == RT_OK) {
    rt_fields3 f3;
    f3.T_K = fields->T_K;
    f3.n_h2_cm3 = fields->n_h2_cm3;
    f3.vturb = fields->vturb;
    f3.x_co = fields->x_co;
    f3.vx_kms = fields->vr_kms;
    f3.vy_kms = fields->vth_kms;
    f3.vz_kms = fields->vph_kms;
    f3.vturb_mach = fields->vturb_mach;
    rc = adjoint3_call(*P, &f3, nullptr, (long long)grid->nr * grid->nth * grid->nph, dL_dcube,
                       target, cube_out, grads, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_pack_nodes3(const rt_fields3 *fields3, long long nodes, void *records,
                              void *stream) {
  if (!fields3) return set_error(RT_EINVAL, "null argument struct");
  const rt_fields3 &f = *fields3;
  if (!f.T_K || !f.n_h2_cm3 || !f.vturb || !f.x_co || !f.vx_kms || !f.vy_kms || !f.vz_kms)
    return set_error(RT_EINVAL, "null field pointer");
  if (nodes < 1 || nodes > (1LL << 28))
    return set_error(RT_EINVAL, "node count %lld outside 1 .. 2^28", nodes);
  if (!records || (reinterpret_cast<uintptr_t>(records) & 15))
    return set_error(RT_EINVAL, "records must be a 16-byte aligned device pointer");
  float4 *a = static_cast<float4 *>(records);
  const long long nb = (nodes + 255) / 256;
  pack_nodes3_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, (cudaStream_t)stream>>>(
      f, nodes, a, a + nodes);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "node packing: %s", cudaGetErrorString(e));
  clear_error();
  return RT_OK;
}

namespace rtb {

// A 3-D render (P from build_params3_core or build_params_sph_core) from node records packed
// by rt_pack_nodes3.
static int render_packed(MarchParams &P, const void *records, long long nodes, float *cube,
                         cudaStream_t st) {
  const long long n = (long long)P.nx * P.ny * P.nch;
  if (n > 0 && !cube) return set_error(RT_EINVAL, "null cube pointer");
  if (!records || (reinterpret_cast<uintptr_t>(records) & 15))
    return set_error(RT_EINVAL, "records must be a 16-byte aligned device pointer");
  if (n == 0) return RT_OK;
  P.node_a = static_cast<const float4 *>(records);
  P.node_b = P.node_a + nodes;
  return launch_forward(P, cube, st);
}

}  // namespace rtb

extern "C" int rt_render3d_packed(const rt_grid3 *grid3, const void *records, int vturb_mach,
                                  const rt_geom *geom, const rt_view *view, const rt_line *line,
                                  float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params3_core(grid3, vturb_mach, geom, view, line, P);
  if (rc == RT_OK)
    rc = render_packed(*P, records, (long long)grid3->nx * grid3->ny * grid3->nz, cube,
                       (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_sph_packed(const rt_grid_sph *grid, const void *records, int vturb_mach,
                                    const rt_geom *geom, const rt_view *view,
                                    const rt_line *line, float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params_sph_core(grid, vturb_mach, geom, view, line, P);
  if (rc == RT_OK)
    rc = render_packed(*P, records, (long long)grid->nr * grid->nth * grid->nph, cube,
                       (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render3d_adjoint_packed(const rt_grid3 *grid3, const void *records,
                                          int vturb_mach, const rt_geom *geom,
                                          const rt_view *view, const rt_line *line,
                                          const float *dL_dcube, const float *target,
                                          float *cube_out, const rt_grads3 *grads,
                                          void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params3_core(grid3, vturb_mach, geom, view, line, P);
  if (rc == RT_OK && !records) rc = set_error(RT_EINVAL, "null records pointer");
  if (rc == RT_OK)
    rc = adjoint3_call(*P, nullptr, records, (long long)grid3->nx * grid3->ny * grid3->nz,
                       dL_dcube, target, cube_out, grads, (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_sph_adjoint_packed(const rt_grid_sph *grid, const void *records,
                                            int vturb_mach, const rt_geom *geom,
                                            const rt_view *view, const rt_line *line,
                                            const float *dL_dcube, const float *target,
                                            float *cube_out, const rt_grads3 *grads,
                                            void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params_sph_core(grid, vturb_mach, geom, view, line, P);
  if (rc == RT_OK && !records) rc = set_error(RT_EINVAL, "null records pointer");
  if (rc == RT_OK)
    rc = adjoint3_call(*P, nullptr, records, (long long)grid->nr * grid->nth * grid->nph,
                       dL_dcube, target, cube_out, grads, (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                         const rt_view *view, const rt_line *line, float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) {
    long long n = (long long)P->nx * P->ny * P->nch;
    if (n > 0 && !cube)
      rc = set_error(RT_EINVAL, "null cube pointer");
    else
      rc = launch_forward(*P, cube, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_plain(const rt_grid *grid, const rt_fields *fields,
                               const rt_geom *geom, const rt_view *view, const rt_line *line,
                               float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK && P->vphi)
    rc = set_error(RT_EINVAL, "the plain march takes Keplerian rotation only (no vphi_kms)");
  if (rc == RT_OK) {
    const long long n = (long long)P->nx * P->ny * P->nch;
    if (n > 0 && !cube)
      rc = set_error(RT_EINVAL, "null cube pointer");
    else
      rc = launch_plain(*P, cube, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_dense(const rt_grid *grid, const rt_fields *fields,
                               const rt_geom *geom, const rt_view *view, const rt_line *line,
                               float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) {
    const long long n = (long long)P->nx * P->ny * P->nch;
    if (n > 0 && !cube)
      rc = set_error(RT_EINVAL, "null cube pointer");
    else
      rc = launch_forward_dense(*P, cube, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_launch_count(const rt_grid *grid, const rt_fields *fields,
                                      const rt_geom *geom, const rt_view *view,
                                      const rt_line *line, int *count) {
  if (!count) return set_error(RT_EINVAL, "null count pointer");
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) {
    const long long n = (long long)P->nx * P->ny * P->nch;
    *count = n == 0 ? 0 : (cell_bytes(*P) ? 2 : 1);
    clear_error();
  }
  delete P;
  return rc;
}

extern "C" int rt_render_work(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                              const rt_view *view, const rt_line *line, float *cube,
                              unsigned long long *work, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK && !work) rc = set_error(RT_EINVAL, "null work counters");
  if (rc == RT_OK) {
    long long n = (long long)P->nx * P->ny * P->nch;
    cudaError_t e = cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), (cudaStream_t)stream);
    if (e != cudaSuccess) {
      rc = set_error(RT_ECUDA, "memset: %s", cudaGetErrorString(e));
    } else if (n > 0 && !cube) {
      rc = set_error(RT_EINVAL, "null cube pointer");
    } else {
      P->work = work;
      rc = launch_forward(*P, cube, (cudaStream_t)stream);
    }
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_count_gas_samples(const rt_grid *grid, const rt_fields *fields,
                                    const rt_geom *geom, const rt_view *view,
                                    const rt_line *line, unsigned long long *count,
                                    void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) {
    if (!count)
      rc = set_error(RT_EINVAL, "null count pointer");
    else
      rc = launch_count(*P, count, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

// Shared validation of the adjoint seeds and gradient outputs.
int rtb::check_adjoint_args(const MarchParams &P, const float *dL_dcube, const float *target,
                       const rt_grads *grads) {
  if (!grads || !grads->dT || !grads->dn || !grads->dvt || !grads->dh_lo || !grads->dh_hi)
    return set_error(RT_EINVAL, "null gradient output");
  if (P.vphi && !grads->dvphi)
    return set_error(RT_EINVAL, "a rotation field needs its gradient output (grads->dvphi)");
  long long n = (long long)P.nx * P.ny * P.nch;
  if (n > 0 && ((dL_dcube == nullptr) == (target == nullptr)))
    return set_error(RT_EINVAL, "give exactly one of dL_dcube and target");
  return RT_OK;
}

extern "C" int rt_render_adjoint_work(const rt_grid *grid, const rt_fields *fields,
                                      const rt_geom *geom, const rt_view *view,
                                      const rt_line *line, const float *dL_dcube,
                                      const float *target, float *cube_out,
                                      const rt_grads *grads, unsigned long long *work,
                                      void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) rc = check_adjoint_args(*P, dL_dcube, target, grads);
  if (rc == RT_OK && !work) rc = set_error(RT_EINVAL, "null work counters");
  if (rc == RT_OK) {
    cudaError_t e = cudaMemsetAsync(work, 0, 4 * sizeof(unsigned long long), (cudaStream_t)stream);
    if (e != cudaSuccess) rc = set_error(RT_ECUDA, "memset: %s", cudaGetErrorString(e));
  }
  if (rc == RT_OK) {
    P->work = work;
    rc = launch_adjoint(*P, dL_dcube, target, cube_out, *grads, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_adjoint(const rt_grid *grid, const rt_fields *fields,
                                 const rt_geom *geom, const rt_view *view, const rt_line *line,
                                 const float *dL_dcube, const float *target, float *cube_out,
                                 const rt_grads *grads, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) rc = check_adjoint_args(*P, dL_dcube, target, grads);
  if (rc == RT_OK)
    rc = launch_adjoint(*P, dL_dcube, target, cube_out, *grads, (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_pressure_vphi(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                                const float *n_h2, const float *T_K, float *vphi_kms,
                                void *stream) {
  if (!grid || !geom || !line || !n_h2 || !T_K || !vphi_kms)
    return set_error(RT_EINVAL, "null argument");
  if (grid->nr < 2 || grid->nz < 2) return set_error(RT_EINVAL, "grid needs >= 2 nodes per axis");
  if (!(grid->r_in_au > 0) || !(grid->r_out_au > grid->r_in_au) || !(grid->zr_max > 0) ||
      !is_finite(grid->r_out_au) || !is_finite(grid->zr_max))
    return set_error(RT_EINVAL, "invalid grid extent");
  if (!(geom->mstar_msun >= 0) || !is_finite(geom->mstar_msun))
    return set_error(RT_EINVAL, "stellar mass must be finite and >= 0");
  if (!(line->m_mol_amu > 0) || !is_finite(line->m_mol_amu))
    return set_error(RT_EINVAL, "mean molecular mass must be > 0");
  int rc = launch_pressure_vphi(*grid, *geom, *line, n_h2, T_K, vphi_kms, (cudaStream_t)stream);
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_pressure_vphi_adjoint(const rt_grid *grid, const rt_geom *geom,
                                        const rt_line *line, const float *n_h2,
                                        const float *T_K, const double *g_vphi, double *g_n,
                                        double *g_T, void *stream) {
  if (!grid || !geom || !line || !n_h2 || !T_K || !g_vphi || !g_n || !g_T)
    return set_error(RT_EINVAL, "null argument");
  if (grid->nr < 2 || grid->nz < 2) return set_error(RT_EINVAL, "grid needs >= 2 nodes per axis");
  if (!(grid->r_in_au > 0) || !(grid->r_out_au > grid->r_in_au) || !(grid->zr_max > 0) ||
      !is_finite(grid->r_out_au) || !is_finite(grid->zr_max))
    return set_error(RT_EINVAL, "invalid grid extent");
  if (!(geom->mstar_msun >= 0) || !is_finite(geom->mstar_msun))
    return set_error(RT_EINVAL, "stellar mass must be finite and >= 0");
  if (!(line->m_mol_amu > 0) || !is_finite(line->m_mol_amu))
    return set_error(RT_EINVAL, "mean molecular mass must be > 0");
  int rc = launch_pressure_vphi_adjoint(*grid, *geom, *line, n_h2, T_K, g_vphi, g_n, g_T,
                                        (cudaStream_t)stream);
  if (rc == RT_OK) clear_error();
  return rc;
}

static int check_chain_args(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                            const rt_chain *chain) {
  if (grid->nr < 2 || grid->nz < 2) return set_error(RT_EINVAL, "grid needs >= 2 nodes per axis");
  if (!(grid->r_in_au > 0) || !(grid->r_out_au > grid->r_in_au) || !(grid->zr_max > 0) ||
      !is_finite(grid->r_out_au) || !is_finite(grid->zr_max))
    return set_error(RT_EINVAL, "invalid grid extent");
  if (!(geom->mstar_msun >= 0) || !is_finite(geom->mstar_msun))
    return set_error(RT_EINVAL, "stellar mass must be finite and >= 0");
  if (!(line->m_mol_amu > 0) || !is_finite(line->m_mol_amu))
    return set_error(RT_EINVAL, "mean molecular mass must be > 0");
  if (!(chain->sigma0_gcm2 >= 0) || !is_finite(chain->sigma0_gcm2) || !(chain->r_c_au > 0) ||
      !is_finite(chain->r_c_au) || !(chain->gamma < 2) || !is_finite(chain->gamma) ||
      !is_finite(chain->T_freeze_K) || !(chain->N_dissoc_cm2 >= 0) ||
      !is_finite(chain->N_dissoc_cm2))
    return set_error(RT_EINVAL, "invalid chain parameters");
  return RT_OK;
}

extern "C" int rt_field_chain_adjoint(const rt_grid *grid, const rt_geom *geom,
                                      const rt_line *line, const rt_chain *chain,
                                      const float *T_K, const double *g_n,
                                      const double *g_lo, const double *g_hi, double *g_T,
                                      void *stream) {
  if (!grid || !geom || !line || !chain || !T_K || !g_T)
    return set_error(RT_EINVAL, "null argument");
  int rc = check_chain_args(grid, geom, line, chain);
  if (rc != RT_OK) return rc;
  rc = launch_field_chain_adjoint(*grid, *geom, *line, *chain, T_K, g_n, g_lo, g_hi, g_T,
                                  (cudaStream_t)stream);
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_field_chain(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                              const rt_chain *chain, const float *T_K, float *n_h2,
                              float *N_h2, float *h_lo, float *h_hi, void *stream) {
  if (!grid || !geom || !line || !chain || !T_K || !n_h2 || !h_lo || !h_hi)
    return set_error(RT_EINVAL, "null argument");
  if (grid->nr < 2 || grid->nz < 2) return set_error(RT_EINVAL, "grid needs >= 2 nodes per axis");
  if (!(grid->r_in_au > 0) || !(grid->r_out_au > grid->r_in_au) || !(grid->zr_max > 0) ||
      !is_finite(grid->r_out_au) || !is_finite(grid->zr_max))
    return set_error(RT_EINVAL, "invalid grid extent");
  if (!(geom->mstar_msun >= 0) || !is_finite(geom->mstar_msun))
    return set_error(RT_EINVAL, "stellar mass must be finite and >= 0");
  if (!(line->m_mol_amu > 0) || !is_finite(line->m_mol_amu))
    return set_error(RT_EINVAL, "mean molecular mass must be > 0");
  if (!(chain->sigma0_gcm2 >= 0) || !is_finite(chain->sigma0_gcm2) || !(chain->r_c_au > 0) ||
      !is_finite(chain->r_c_au) || !(chain->gamma < 2) || !is_finite(chain->gamma) ||
      !is_finite(chain->T_freeze_K) || !(chain->N_dissoc_cm2 >= 0) ||
      !is_finite(chain->N_dissoc_cm2))
    return set_error(RT_EINVAL, "invalid chain parameters");
  int rc = launch_field_chain(*grid, *geom, *line, *chain, T_K, n_h2, N_h2, h_lo, h_hi,
                              (cudaStream_t)stream);
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_surface_powerlaw_grad(const rt_grid *grid, const double *dh, const float *h,
                                        double c, double *out, void *stream) {
  if (!grid || !dh || !h || !out) return set_error(RT_EINVAL, "null argument");
  if (grid->nr < 2 || !(grid->r_in_au > 0) || !(grid->r_out_au > grid->r_in_au))
    return set_error(RT_EINVAL, "invalid grid");
  if (!is_finite(c) || c == 0.0) return set_error(RT_EINVAL, "surface coefficient must be non-zero");
  int rc = launch_surface_grad(*grid, dh, h, c, out, (cudaStream_t)stream);
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_sample_coords(const rt_grid *grid, const rt_fields *fields,
                                const rt_geom *geom, const rt_view *view, const rt_line *line,
                                float *xy, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK && (long long)P->nx * P->ny > 0 && !xy) rc = set_error(RT_EINVAL, "null output");
  if (rc == RT_OK) rc = launch_coords(*P, reinterpret_cast<float2 *>(xy), (cudaStream_t)stream);
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_modulated(const rt_grid *grid, const rt_fields *fields,
                                   const rt_geom *geom, const rt_view *view, const rt_line *line,
                                   const float *mod, double h_scale, float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  long long n = rc == RT_OK ? (long long)P->nx * P->ny * P->nch : 0;
  if (rc == RT_OK && n > 0 && (!cube || !mod)) rc = set_error(RT_EINVAL, "null cube or modulation");
  if (rc == RT_OK && !is_finite(h_scale)) rc = set_error(RT_EINVAL, "non-finite h_scale");
  if (rc == RT_OK) {
    P->mod = reinterpret_cast<const float4 *>(mod);
    P->h_scale = (float)h_scale;
    rc = launch_forward(*P, cube, (cudaStream_t)stream);
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_mlp(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                             const rt_view *view, const rt_line *line, const rt_mlp *mlp,
                             float *cube, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) rc = mlp_validate(mlp);
  long long npix = rc == RT_OK ? (long long)P->nx * P->ny : 0;
  if (rc == RT_OK && npix * P->nch > 0 && !cube) rc = set_error(RT_EINVAL, "null cube pointer");
  if (rc == RT_OK && npix * P->nch > 0) {
    cudaStream_t st = (cudaStream_t)stream;
    size_t mod_bytes = (size_t)npix * P->n_samples * sizeof(float4);
    size_t ray_bytes = (ray_buffer_bytes(npix) + 255) & ~(size_t)255;
    size_t list_bytes = sample_list_bytes(npix, P->n_samples);
    size_t bytes = mod_bytes + ray_bytes + list_bytes;
    float4 *mod = nullptr;
    cudaError_t e = stream_alloc((void **)&mod, bytes, st);
    if (e != cudaSuccess) {
      rc = set_error(RT_ENOMEM, "modulation buffer (%zu bytes): %s", bytes, cudaGetErrorString(e));
    } else {
      char *rays = reinterpret_cast<char *>(mod) + mod_bytes;
      rc = launch_mlp_rays(mlp, *P, mod, rays, list_bytes ? rays + ray_bytes : nullptr, st);
      if (rc == RT_OK) {
        P->mod = mod;
        P->h_scale = (float)mlp->h_scale;
        rc = launch_forward(*P, cube, st);
      }
      cudaFreeAsync(mod, st);
    }
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_render_mlp_adjoint(const rt_grid *grid, const rt_fields *fields,
                                     const rt_geom *geom, const rt_view *view,
                                     const rt_line *line, const rt_mlp *mlp,
                                     const float *dL_dcube, const float *target,
                                     float *cube_out, const rt_grads *grads,
                                     const rt_mlp_grads *mlp_grads, void *stream) {
  MarchParams *P = new (std::nothrow) MarchParams;
  if (!P) return set_error(RT_ENOMEM, "host allocation failed");
  int rc = build_params(grid, fields, geom, view, line, P);
  if (rc == RT_OK) rc = mlp_validate(mlp);
  if (rc == RT_OK) rc = mlp_grads_validate(mlp_grads);
  if (rc == RT_OK) rc = check_adjoint_args(*P, dL_dcube, target, grads);
  const long long npix = rc == RT_OK ? (long long)P->nx * P->ny : 0;
  const long long ns = npix * (rc == RT_OK ? P->n_samples : 0);
  if (rc == RT_OK) {
    cudaStream_t st = (cudaStream_t)stream;
    // one buffer: network outputs (after the march adjoint: the gathered output gradients of
    // the backward), dL/d(outputs), ray setups, sample list, gathered network inputs, backward
    // scratch, gradient scale
    const size_t ng = mlp_bwd_gather_entries(ns);
    const size_t mod_bytes = ((ng > (size_t)ns ? ng : (size_t)ns) * sizeof(float4) + 255) & ~(size_t)255;
    const size_t ray_bytes = (ray_buffer_bytes(npix) + 255) & ~(size_t)255;
    const size_t list_bytes = (sample_list_bytes(npix, P->n_samples) + 255) & ~(size_t)255;
    const size_t xy_bytes = (ng * sizeof(float2) + 255) & ~(size_t)255;
    const size_t spill_bytes = mlp_bwd_scratch_bytes(ns);
    const size_t bytes = 2 * mod_bytes + ray_bytes + list_bytes + xy_bytes + spill_bytes + 256;
    char *buf = nullptr;
    cudaError_t e = stream_alloc((void **)&buf, bytes, st);
    if (e != cudaSuccess) {
      rc = set_error(RT_ENOMEM, "neural adjoint buffers (%zu bytes): %s", bytes,
                     cudaGetErrorString(e));
    } else {
      float4 *mod = reinterpret_cast<float4 *>(buf);
      float4 *dmod = reinterpret_cast<float4 *>(buf + mod_bytes);
      char *rays = buf + 2 * mod_bytes;
      char *list = list_bytes ? rays + ray_bytes : nullptr;
      float2 *xy = reinterpret_cast<float2 *>(rays + ray_bytes + list_bytes);
      char *spill = rays + ray_bytes + list_bytes + xy_bytes;
      unsigned *dmax = reinterpret_cast<unsigned *>(spill + spill_bytes);
      e = cudaMemsetAsync(dmod, 0, mod_bytes, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, sizeof(unsigned), st);
      if (e != cudaSuccess) rc = set_error(RT_ECUDA, "memset: %s", cudaGetErrorString(e));
      if (rc == RT_OK && ns > 0) rc = launch_mlp_rays(mlp, *P, mod, rays, list, st);
      if (rc == RT_OK) {
        P->mod = ns > 0 ? mod : nullptr;
        P->h_scale = (float)mlp->h_scale;
        rc = launch_adjoint(*P, dL_dcube, target, cube_out, *grads, st, dmod, dmax);
      }
      if (rc == RT_OK)
        rc = launch_mlp_bwd_rays(mlp, *P, rays, ns > 0 ? list : nullptr, dmod, dmax, spill, xy,
                                 mod, mlp_grads, st);
      cudaFreeAsync(buf, st);
    }
  }
  delete P;
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" const char *rt_last_error(void) { return g_err; }

extern "C" const char *rt_version(void) { return "b300-linert 0.1 (sm_103a)"; }
