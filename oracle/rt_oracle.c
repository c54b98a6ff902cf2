/*
 * FP64 CPU oracle for the line radiative-transfer march -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow and deliberately unoptimised: every step is written in the order and notation
 * of arXiv 2509.03623, Methods, "Line Radiative Transfer with RadJAX":
 *   I_nu = int j_nu(s') exp(-tau_nu(s,s')) ds'          (Eq. rt-int)
 *   tau_nu(s,s') = int_{s'}^{s} beta_nu ds''             (Eq. optical_depth)
 *   j_nu    = h nu0/(4 pi) n_u A_ul phi                  (emissivity equation)
 *   beta_nu = h nu0/(4 pi) (n_l B_lu - n_u B_ul) phi     (extinction equation)
 *   phi(nu) = c/(nu0 alpha sqrt(pi)) exp(-(c[nu - nu0(1-dnu)]/(nu0 alpha))^2),
 *             dnu = omega.v/c                            (line-profile equation)
 *   alpha   = sqrt(2kT/m_CO + v_turb^2 c_s^2), c_s^2 = 2kT/m_mol (line-width equations)
 *   v_phi^2/r = G M r/(r^2+z^2)^{3/2}                    (Keplerian term of
 *                                                          Eq. gas_velocity_pressure)
 * with LTE (Boltzmann) populations of a rigid rotor. Where the paper is silent the readings
 * are stated at the point of use (sampling rule, grid interpolation, CO-layer edges, sign and
 * frame conventions); the design notes list them all.
 *
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may load this file.
 * It shares nothing with the CUDA library.
 */
#include "rt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* CGS constants: CODATA 2018 exact SI-defining values, IAU 2012/2015 nominal values. */
static const double H_PLANCK = 6.62607015e-27;  /* erg s */
static const double K_BOLTZ = 1.380649e-16;     /* erg K^-1 */
static const double C_LIGHT = 2.99792458e10;    /* cm s^-1 */
static const double AMU_G = 1.66053906660e-24;  /* g */
static const double GM_SUN = 1.3271244e26;      /* cm^3 s^-2, IAU 2015 nominal */
static const double AU_CM = 1.495978707e13;     /* cm, IAU 2012 */
/* 1 au at 1 pc subtends 1 arcsec (definition of the parsec). */
static const double ARCSEC_RAD = M_PI / 648000.0;

/* ---------------------------------------------------------------------------------------- */
/* Molecular data: LTE rigid rotor (the paper precomputes Boltzmann populations from       */
/* tabulated levels; the table is replaced by E_J = h B J(J+1), g_J = 2J+1).                */
/* ---------------------------------------------------------------------------------------- */

static double rot_B(const orc_problem *p) {
  return p->B_rot_hz > 0 ? p->B_rot_hz : p->nu0_hz / (2.0 * p->J_u);
}

double orc_partition(double T, double B_rot_hz) {
  /* Z(T) = sum_J (2J+1) exp(-h B J(J+1)/kT), summed until the term is below 1e-17 Z. */
  double Z = 0.0;
  for (int J = 0; J < 100000; J++) {
    double term = (2.0 * J + 1.0) * exp(-H_PLANCK * B_rot_hz * J * (J + 1.0) / (K_BOLTZ * T));
    Z += term;
    if (J > 2 && term < 1e-17 * Z) break;
  }
  return Z;
}

/* Mean level energy <E> = sum g E exp(-E/kT) / Z (for dZ/dT = Z <E>/(k T^2)). */
static double mean_energy(double T, double B) {
  double Z = 0.0, EZ = 0.0;
  for (int J = 0; J < 100000; J++) {
    double E = H_PLANCK * B * J * (J + 1.0);
    double term = (2.0 * J + 1.0) * exp(-E / (K_BOLTZ * T));
    Z += term;
    EZ += E * term;
    if (J > 2 && term < 1e-17 * Z) break;
  }
  return EZ / Z;
}

/* ---------------------------------------------------------------------------------------- */
/* Geometry                                                                                */
/* ---------------------------------------------------------------------------------------- */

static double box_reach(const orc_grid3 *g) {
  double m = fmax(fmax(fabs(g->x0), fabs(g->x1)), fmax(fabs(g->y0), fabs(g->y1)));
  return fmax(m, fmax(fabs(g->z0), fabs(g->z1)));
}

static double half_fov(const orc_problem *p) {
  if (p->half_fov_au > 0) return p->half_fov_au;
  if (p->gs) return 1.1 * p->gs->r_out;
  return 1.1 * (p->g3 ? box_reach(p->g3) : p->r_out_au);
}

/* Ray through pixel (ix, iy). Disk frame: +z along the disk angular momentum. Observer
   direction n_obs = (0, -sin i, cos i); sky basis e_x = (1,0,0), e_y = (0, cos i, sin i)
   (e_x x e_y = n_obs). Pixel centres (i + 1/2 - n/2) * 2 half_fov / n au; the position
   angle rotates image coordinates into the sky basis. The ray direction omega = -n_obs
   points away from the observer (backward ray tracing), so s increases front to back. */
static void ray_setup(const orc_problem *p, int ix, int iy, double P0[3], double om[3]) {
  double hf = half_fov(p);
  double X = (ix + 0.5 - 0.5 * p->nx) * (2.0 * hf / p->nx);
  double Y = (iy + 0.5 - 0.5 * p->ny) * (2.0 * hf / p->ny);
  double pa = p->pa_deg * M_PI / 180.0, inc = p->incl_deg * M_PI / 180.0;
  double xs = X * cos(pa) + Y * sin(pa);
  double ys = -X * sin(pa) + Y * cos(pa);
  double ex[3] = {1.0, 0.0, 0.0};
  double ey[3] = {0.0, cos(inc), sin(inc)};
  double nobs[3] = {0.0, -sin(inc), cos(inc)};
  for (int a = 0; a < 3; a++) {
    P0[a] = xs * ex[a] + ys * ey[a];
    om[a] = -nobs[a];
  }
}

/* Chord of the ray through the bounding cylinder r <= r_out, |z| <= zr_max r_out
   (sampling rule: the paper does not state one). */
static int chord(const orc_problem *p, const double P0[3], const double om[3], double *s0,
                 double *s1) {
  if (p->gs) {
    /* spherical grid: the chord through the sphere r <= r_out, |P0 + s om| = r_out with
       |om| = 1 */
    const double R = p->gs->r_out;
    const double b = P0[0] * om[0] + P0[1] * om[1] + P0[2] * om[2];
    const double c = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2] - R * R;
    const double disc = b * b - c;
    if (!(disc > 0.0)) return 0;
    *s0 = -b - sqrt(disc);
    *s1 = -b + sqrt(disc);
    return 1;
  }
  if (p->g3) {
    /* 3-D grid: the chord through the box, slab by slab */
    const double lo3[3] = {p->g3->x0, p->g3->y0, p->g3->z0};
    const double hi3[3] = {p->g3->x1, p->g3->y1, p->g3->z1};
    double lo = -INFINITY, hi = INFINITY;
    for (int a = 0; a < 3; a++) {
      if (om[a] != 0.0) {
        double t1 = (lo3[a] - P0[a]) / om[a], t2 = (hi3[a] - P0[a]) / om[a];
        lo = fmax(lo, fmin(t1, t2));
        hi = fmin(hi, fmax(t1, t2));
      } else if (P0[a] < lo3[a] || P0[a] > hi3[a]) {
        return 0;
      }
    }
    if (!(hi > lo)) return 0;
    *s0 = lo;
    *s1 = hi;
    return 1;
  }
  double R = p->r_out_au, H = p->zr_max * p->r_out_au;
  double lo = -INFINITY, hi = INFINITY;
  if (om[2] != 0.0) {
    double t1 = (-H - P0[2]) / om[2], t2 = (H - P0[2]) / om[2];
    lo = fmax(lo, fmin(t1, t2));
    hi = fmin(hi, fmax(t1, t2));
  } else if (fabs(P0[2]) > H) {
    return 0;
  }
  double a = om[0] * om[0] + om[1] * om[1];
  double b = 2.0 * (P0[0] * om[0] + P0[1] * om[1]);
  double c = P0[0] * P0[0] + P0[1] * P0[1] - R * R;
  if (a > 0.0) {
    /* b^2 - 4ac; for a ray of constant x (om[0] = 0, every view of the disk) it equals
       4a (R - x)(R + x), evaluated so: the difference of squares loses the chords of rays
       that graze the wall */
    double disc = om[0] == 0.0 ? 4.0 * a * ((R - P0[0]) * (R + P0[0])) : b * b - 4.0 * a * c;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    lo = fmax(lo, (-b - sq) / (2.0 * a));
    hi = fmin(hi, (-b + sq) / (2.0 * a));
  } else if (c > 0.0) {
    return 0;
  }
  if (!(hi > lo)) return 0;
  *s0 = lo;
  *s1 = hi;
  return 1;
}

int orc_ray(const orc_problem *p, int ix, int iy, double *s_in, double *s_out, double *P0,
            double *omega) {
  double P[3], om[3];
  ray_setup(p, ix, iy, P, om);
  for (int a = 0; a < 3; a++) {
    P0[a] = P[a];
    omega[a] = om[a];
  }
  return chord(p, P, om, s_in, s_out);
}

/* ---------------------------------------------------------------------------------------- */
/* Local state at a point                                                                  */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
  int gas;
  /* interpolation: r-cell i0 with weight fr, (z/r)-cell j0 with weight fz */
  int i0, j0;
  double fr, fz;
  double zr;                  /* |z|/r */
  double T, n, vt, hlo, hhi;  /* interpolated primitives */
  double sa, sb, X;           /* CO-layer edge factors and abundance */
  double vlos;                /* cm/s, positive receding */
  double alpha;               /* cm/s */
  double Z, fu, fl;           /* partition function, n_u/n_CO, n_l/n_CO */
  double nco, nu_, nl_;       /* n_CO, n_u, n_l */
  double D;                   /* n_l B_lu - n_u B_ul */
  double S;                   /* j/beta */
  /* neural field (when a network is given): inputs, outputs and the factors exp(o0), exp(o1)
     applied to T and n */
  double xin[2], o[4], mT, mn;
  /* d v_los / d(rotation-field value) [cm/s per km/s] with a rotation field, 0 otherwise */
  double dvlos_dvphi;
  /* 3-D grids: the cell (lowest node index per axis; on the spherical grid k1 is the azimuth
     node after i3[2], periodic) and the fractional position in it, as the trilinear
     interpolation used them, and d v_los / d(the three velocity fields) [cm/s per km/s] */
  int i3[3], k1;
  double f3[3], dv3[3];
} pt;

static double bilerp(const double *F, int nr, int i0, int j0, double fr, double fz) {
  return (1.0 - fr) * (1.0 - fz) * F[j0 * nr + i0] + fr * (1.0 - fz) * F[j0 * nr + i0 + 1] +
         (1.0 - fr) * fz * F[(j0 + 1) * nr + i0] + fr * fz * F[(j0 + 1) * nr + i0 + 1];
}

static double logistic(double x) { return 1.0 / (1.0 + exp(-x)); }

#define ORC_MLP_MAXW 1024

static void mlp_forward(const orc_mlp *m, const double xin[2], double *out);

/* Evaluate the local state at disk-frame point P (au). */
static void eval_point(const orc_problem *p, const orc_mlp *m, const double P[3],
                       const double om[3], pt *st) {
  memset(st, 0, sizeof(*st));
  double x = P[0], y = P[1], z = P[2];
  if (p->gs) {
    /* spherical grid: (r, theta, phi) of the point, trilinear interpolation (periodic in
       phi), the gas velocity from its spherical components */
    const orc_grid_sph *g = p->gs;
    const double Rc = sqrt(x * x + y * y), r = sqrt(Rc * Rc + z * z);
    if (!(r >= g->r_in && r <= g->r_out)) return;
    const double th = atan2(Rc, z);
    if (!(th >= g->th0 && th <= g->th1)) return;
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * M_PI;
    double u = g->r_log ? log(r / g->r_in) / log(g->r_out / g->r_in) * (g->nr - 1)
                        : (r - g->r_in) / (g->r_out - g->r_in) * (g->nr - 1);
    double v = (th - g->th0) / (g->th1 - g->th0) * (g->nth - 1);
    double w = ph / (2.0 * M_PI) * g->nph;
    if (u > g->nr - 1) u = g->nr - 1;
    if (u < 0) u = 0;
    if (v > g->nth - 1) v = g->nth - 1;
    if (v < 0) v = 0;
    int i0 = (int)floor(u), j0 = (int)floor(v), k0 = (int)floor(w);
    if (i0 > g->nr - 2) i0 = g->nr - 2;
    if (j0 > g->nth - 2) j0 = g->nth - 2;
    const double f[3] = {u - i0, v - j0, w - k0};
    k0 %= g->nph;
    const int k1 = (k0 + 1) % g->nph;
    const double *F[7] = {g->T, g->n_h2, g->vturb, g->x_co, g->vr, g->vth, g->vph};
    double val[7];
    for (int q = 0; q < 7; q++) {
      double acc = 0.0;
      for (int c = 0; c < 8; c++) {
        const int di = c & 1, dj = (c >> 1) & 1, dk = c >> 2;
        const double wt = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) *
                          (dk ? f[2] : 1.0 - f[2]);
        acc += wt * F[q][((long long)(dk ? k1 : k0) * g->nth + (j0 + dj)) * g->nr + (i0 + di)];
      }
      val[q] = acc;
    }
    st->T = val[0];
    st->n = val[1];
    st->vt = val[2];
    st->X = val[3];
    /* unit vectors r^ = (x, y, z)/r, theta^ = (cos th cos ph, cos th sin ph, -sin th),
       phi^ = (-sin ph, cos ph, 0); on the axis (Rc = 0) theta^ and phi^ are taken as 0, and
       at the centre (r = 0) r^ as well */
    const double st_ = r > 0 ? Rc / r : 0.0, ct = r > 0 ? z / r : 0.0;
    const double cp = Rc > 0 ? x / Rc : 0.0, sp = Rc > 0 ? y / Rc : 0.0;
    const double vel[3] = {val[4] * st_ * cp + val[5] * ct * cp - val[6] * sp,
                           val[4] * st_ * sp + val[5] * ct * sp + val[6] * cp,
                           val[4] * ct - val[5] * st_};
    st->i3[0] = i0;
    st->i3[1] = j0;
    st->i3[2] = k0;
    st->k1 = k1;
    for (int a = 0; a < 3; a++) st->f3[a] = f[a];
    /* v_los = 1e5 omega . (v_r r^ + v_theta theta^ + v_phi phi^) + v_sys */
    st->dv3[0] = 1e5 * (om[0] * st_ * cp + om[1] * st_ * sp + om[2] * ct);
    st->dv3[1] = 1e5 * (om[0] * ct * cp + om[1] * ct * sp - om[2] * st_);
    st->dv3[2] = 1e5 * (-om[0] * sp + om[1] * cp);
    st->vlos = 1e5 * (om[0] * vel[0] + om[1] * vel[1] + om[2] * vel[2]) + p->vsys_kms * 1e5;
    goto line_physics;
  }
  if (p->g3) {
    /* 3-D grid: trilinear interpolation of every field, the abundance from its own field and
       the line-of-sight velocity from the gas velocity field */
    const orc_grid3 *g = p->g3;
    if (x < g->x0 || x > g->x1 || y < g->y0 || y > g->y1 || z < g->z0 || z > g->z1) return;
    double f[3] = {(x - g->x0) / (g->x1 - g->x0) * (g->nx - 1),
                   (y - g->y0) / (g->y1 - g->y0) * (g->ny - 1),
                   (z - g->z0) / (g->z1 - g->z0) * (g->nz - 1)};
    const int nn[3] = {g->nx, g->ny, g->nz};
    int i3[3];
    for (int a = 0; a < 3; a++) {
      i3[a] = (int)floor(f[a]);
      if (i3[a] > nn[a] - 2) i3[a] = nn[a] - 2;
      if (i3[a] < 0) i3[a] = 0;
      f[a] -= i3[a];
    }
    const double *F[7] = {g->T, g->n_h2, g->vturb, g->x_co, g->vx, g->vy, g->vz};
    double val[7];
    for (int q = 0; q < 7; q++) {
      double acc = 0.0;
      for (int c = 0; c < 8; c++) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        acc += w * F[q][((long long)(i3[2] + dz) * g->ny + (i3[1] + dy)) * g->nx + (i3[0] + dx)];
      }
      val[q] = acc;
    }
    for (int a = 0; a < 3; a++) {
      st->i3[a] = i3[a];
      st->f3[a] = f[a];
      st->dv3[a] = 1e5 * om[a];
    }
    st->T = val[0];
    st->n = val[1];
    st->vt = val[2];
    st->X = val[3];
    st->vlos = 1e5 * (om[0] * val[4] + om[1] * val[5] + om[2] * val[6]) + p->vsys_kms * 1e5;
    goto line_physics;
  }
  {
  double r = sqrt(x * x + y * y);
  double zr = r > 0 ? fabs(z) / r : INFINITY;
  st->zr = zr;
  /* Outside the grid (reading): r < r_in or z/r > zr_max carries no gas. */
  if (!(r >= p->r_in_au) || !(zr <= p->zr_max)) return;
  /* Fractional node coordinates: log-spaced (or linear) in r, linear in z/r; clamped to
     the last cell. */
  double u;
  if (p->r_log)
    u = (log(r) - log(p->r_in_au)) / (log(p->r_out_au) - log(p->r_in_au)) * (p->nr - 1);
  else
    u = (r - p->r_in_au) / (p->r_out_au - p->r_in_au) * (p->nr - 1);
  if (u > p->nr - 1) u = p->nr - 1;
  if (u < 0) u = 0;
  int i0 = (int)floor(u);
  if (i0 > p->nr - 2) i0 = p->nr - 2;
  double w = zr / p->zr_max * (p->nz - 1);
  if (w > p->nz - 1) w = p->nz - 1;
  int j0 = (int)floor(w);
  if (j0 > p->nz - 2) j0 = p->nz - 2;
  st->i0 = i0;
  st->j0 = j0;
  st->fr = u - i0;
  st->fz = w - j0;
  /* Bilinear interpolation of the primitive fields (mirror symmetry: |z|). */
  st->T = bilerp(p->T, p->nr, i0, j0, st->fr, st->fz);
  st->n = bilerp(p->n_h2, p->nr, i0, j0, st->fr, st->fz);
  st->vt = bilerp(p->vturb, p->nr, i0, j0, st->fr, st->fz);
  st->hlo = (1.0 - st->fr) * p->h_lo[i0] + st->fr * p->h_lo[i0 + 1];
  st->hhi = (1.0 - st->fr) * p->h_hi[i0] + st->fr * p->h_hi[i0 + 1];
  if (m) {
    /* Neural field: outputs modulate the grid fields (log T, log n residuals and surface
       offsets). Inputs are the normalised grid coordinates. */
    double xin[2] = {u / (p->nr - 1), zr / p->zr_max};
    double o[64];
    mlp_forward(m, xin, o);
    st->xin[0] = xin[0];
    st->xin[1] = xin[1];
    for (int a = 0; a < 4; a++) st->o[a] = o[a];
    st->mT = exp(o[0]);
    st->mn = exp(o[1]);
    st->T *= st->mT;
    st->n *= st->mn;
    st->hlo += m->h_scale * o[2];
    st->hhi += m->h_scale * o[3];
  } else {
    st->mT = st->mn = 1.0;
  }
  /* CO layer between the two surfaces (stand-in for the freeze-out / photodissociation
     gates of Eq. co_layer): logistic edges of width edge_w in z/r, or hard steps. */
  if (p->edge_w > 0) {
    st->sa = logistic((zr - st->hlo) / p->edge_w);
    st->sb = logistic((st->hhi - zr) / p->edge_w);
  } else {
    st->sa = zr >= st->hlo ? 1.0 : 0.0;
    st->sb = zr <= st->hhi ? 1.0 : 0.0;
  }
  st->X = p->x_co * st->sa * st->sb;
  /* Keplerian rotation (first term of Eq. gas_velocity_pressure), counter-clockwise about
     +z: v = v_phi (-y/r, x/r, 0). Line-of-sight velocity omega.v plus systemic velocity. */
  double rc = r * AU_CM, zc = z * AU_CM;
  /* with a rotation field (pressure-corrected, Eq. gas_velocity_pressure): its bilinear
     interpolation, km/s -> cm/s */
  double vphi = p->vphi ? 1e5 * bilerp(p->vphi, p->nr, i0, j0, st->fr, st->fz)
                        : sqrt(GM_SUN * p->mstar_msun * rc * rc / pow(rc * rc + zc * zc, 1.5));
  double v[3] = {-vphi * y / r, vphi * x / r, 0.0};
  st->vlos = om[0] * v[0] + om[1] * v[1] + om[2] * v[2] + p->vsys_kms * 1e5;
  st->dvlos_dvphi = p->vphi ? 1e5 * (om[1] * x - om[0] * y) / r : 0.0;
  }
line_physics:;
  /* Line width: thermal + turbulent. Absolute mode (v_turb in km/s) or the paper's Mach
     form with c_s^2 = 2kT/m_mol as printed. */
  double mco = p->m_co_amu * AMU_G, mmol = p->m_mol_amu * AMU_G;
  double th = 2.0 * K_BOLTZ * st->T / mco;
  if (p->vturb_mach)
    st->alpha = sqrt(th + st->vt * st->vt * (2.0 * K_BOLTZ * st->T / mmol));
  else
    st->alpha = sqrt(th + (st->vt * 1e5) * (st->vt * 1e5));
  /* LTE Boltzmann populations. */
  double B = rot_B(p);
  int Ju = p->J_u, Jl = p->J_u - 1;
  double Eu = H_PLANCK * B * Ju * (Ju + 1.0), El = H_PLANCK * B * Jl * (Jl + 1.0);
  st->Z = orc_partition(st->T, B);
  st->fu = (2.0 * Ju + 1.0) * exp(-Eu / (K_BOLTZ * st->T)) / st->Z;
  st->fl = (2.0 * Jl + 1.0) * exp(-El / (K_BOLTZ * st->T)) / st->Z;
  st->nco = st->X * st->n;
  st->nu_ = st->nco * st->fu;
  st->nl_ = st->nco * st->fl;
  /* Einstein coefficients: B_ul = A_ul c^2/(2 h nu0^3), B_lu = (g_u/g_l) B_ul. */
  double Bul = p->A_ul * C_LIGHT * C_LIGHT / (2.0 * H_PLANCK * pow(p->nu0_hz, 3));
  double Blu = (2.0 * Ju + 1.0) / (2.0 * Jl + 1.0) * Bul;
  st->D = st->nl_ * Blu - st->nu_ * Bul;
  /* Source function S = j/beta; the profile cancels, so it is formed from the
     populations (the pins check it equals the Planck function B_nu0(T)). */
  double Du = st->fl * Blu - st->fu * Bul;
  st->S = p->A_ul * st->fu / Du;
  st->gas = st->nco > 0.0 ? 1 : 0;
}

/* Profile phi(nu_c) [Hz^-1] for channel velocity v_c [km/s] (radio convention
   nu_c = nu0 (1 - v_c/c)); also returns the profile argument xarg. */
static double profile(const orc_problem *p, const pt *st, double v_kms, double *xarg) {
  double nu0 = p->nu0_hz;
  double nu = nu0 * (1.0 - v_kms * 1e5 / C_LIGHT);
  double dnu = st->vlos / C_LIGHT;
  double xx = C_LIGHT * (nu - nu0 * (1.0 - dnu)) / (nu0 * st->alpha);
  if (xarg) *xarg = xx;
  return C_LIGHT / (nu0 * st->alpha * sqrt(M_PI)) * exp(-xx * xx);
}

int orc_point(const orc_problem *p, double x, double y, double z, double v_kms, double *out) {
  double P[3] = {x, y, z}, P0[3], om[3];
  ray_setup(p, 0, 0, P0, om);
  pt st;
  eval_point(p, NULL, P, om, &st);
  for (int a = 0; a < 12; a++) out[a] = 0.0;
  out[2] = st.T;
  out[3] = st.n;
  out[4] = st.X;
  out[5] = st.vlos * 1e-5;
  out[6] = st.alpha * 1e-5;
  out[11] = st.vt;
  if (!st.gas) return 0;
  double phi = profile(p, &st, v_kms, NULL);
  double hnu = H_PLANCK * p->nu0_hz / (4.0 * M_PI);
  out[0] = hnu * st.nu_ * p->A_ul * phi;
  out[1] = hnu * st.D * phi;
  out[7] = st.nu_;
  out[8] = st.nl_;
  out[9] = phi;
  out[10] = st.S;
  return 1;
}

/* ---------------------------------------------------------------------------------------- */
/* The march (Eq. rt-int with Eq. optical_depth), one ray                                  */
/* ---------------------------------------------------------------------------------------- */

static double unit_conv(const orc_problem *p) {
  if (p->units != 1) return 1.0;
  double hf = half_fov(p);
  double ax = (2.0 * hf / p->nx) / p->dist_pc * ARCSEC_RAD;
  double ay = (2.0 * hf / p->ny) / p->dist_pc * ARCSEC_RAD;
  return ax * ay * 1e23; /* erg s^-1 cm^-2 Hz^-1 sr^-1 -> Jy per pixel */
}

/* Front-to-back march of one pixel. The chord is split into n_samples equal segments with
   the source and extinction taken at each midpoint (piecewise-constant step): over segment
   k the intensity gains Tr_k S_k (1 - exp(-dtau_k)) and Tr_{k+1} = Tr_k exp(-dtau_k). The
   background I0 is attenuated by the whole chord. */
static void march_pixel(const orc_problem *p, const orc_mlp *m, int ix, int iy, double *I) {
  double P0[3], om[3], s0, s1;
  ray_setup(p, ix, iy, P0, om);
  double conv = unit_conv(p);
  if (!chord(p, P0, om, &s0, &s1)) {
    for (int c = 0; c < p->nch; c++) I[c] = p->I0;
    return;
  }
  double ds = (s1 - s0) / p->n_samples;
  double ds_cm = ds * AU_CM;
  double hnu = H_PLANCK * p->nu0_hz / (4.0 * M_PI);
  double *Tr = (double *)malloc(sizeof(double) * p->nch);
  double *Ic = (double *)malloc(sizeof(double) * p->nch);
  for (int c = 0; c < p->nch; c++) {
    Tr[c] = 1.0;
    Ic[c] = 0.0;
  }
  for (int k = 0; k < p->n_samples; k++) {
    double s = s0 + (k + 0.5) * ds;
    double P[3] = {P0[0] + s * om[0], P0[1] + s * om[1], P0[2] + s * om[2]};
    pt st;
    eval_point(p, m, P, om, &st);
    if (!st.gas) continue;
    for (int c = 0; c < p->nch; c++) {
      double phi = profile(p, &st, p->v_kms[c], NULL);
      double beta = hnu * st.D * phi;
      double dtau = beta * ds_cm;
      if (!(dtau > 0.0)) continue;
      Ic[c] += Tr[c] * st.S * (-expm1(-dtau));
      Tr[c] *= exp(-dtau);
    }
  }
  for (int c = 0; c < p->nch; c++) I[c] = Ic[c] * conv + p->I0 * Tr[c];
  free(Tr);
  free(Ic);
}

static int check(const orc_problem *p) {
  if (p && p->gs) {
    const orc_grid_sph *g = p->gs;
    if (p->g3 || g->nr < 2 || g->nth < 2 || g->nph < 1 || !(g->r_in >= 0) ||
        !(g->r_out > g->r_in) || (g->r_log && !(g->r_in > 0)) || !(g->th0 >= 0) ||
        !(g->th1 > g->th0) || !(g->th1 <= M_PI) || !g->T || !g->n_h2 || !g->vturb ||
        !g->x_co || !g->vr || !g->vth || !g->vph)
      return -1;
    if (p->nx < 1 || p->ny < 1 || p->nch < 0 || p->n_samples < 1 || (p->nch > 0 && !p->v_kms))
      return -1;
    if (p->J_u < 1 || !(p->nu0_hz > 0) || !(p->dist_pc > 0)) return -1;
    return 0;
  }
  if (p && p->g3) {
    const orc_grid3 *g = p->g3;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || !(g->x1 > g->x0) || !(g->y1 > g->y0) ||
        !(g->z1 > g->z0) || !g->T || !g->n_h2 || !g->vturb || !g->x_co || !g->vx || !g->vy ||
        !g->vz)
      return -1;
    if (p->nx < 1 || p->ny < 1 || p->nch < 0 || p->n_samples < 1 || (p->nch > 0 && !p->v_kms))
      return -1;
    if (p->J_u < 1 || !(p->nu0_hz > 0) || !(p->dist_pc > 0)) return -1;
    return 0;
  }
  if (!p || p->nr < 2 || p->nz < 2 || p->nx < 1 || p->ny < 1 || p->nch < 0 ||
      p->n_samples < 1)
    return -1;
  if (!(p->r_in_au > 0) || !(p->r_out_au > p->r_in_au) || !(p->zr_max > 0)) return -1;
  if (!p->T || !p->n_h2 || !p->vturb || !p->h_lo || !p->h_hi || (p->nch > 0 && !p->v_kms))
    return -1;
  if (p->J_u < 1 || !(p->nu0_hz > 0) || !(p->dist_pc > 0)) return -1;
  return 0;
}

int orc_render(const orc_problem *p, double *cube, int nthreads) {
  if (check(p)) return -1;
  long long npix = (long long)p->nx * p->ny;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int iy = 0; iy < p->ny; iy++) {
    double *I = (double *)malloc(sizeof(double) * (p->nch > 0 ? p->nch : 1));
    for (int ix = 0; ix < p->nx; ix++) {
      march_pixel(p, NULL, ix, iy, I);
      for (int c = 0; c < p->nch; c++) cube[c * npix + (long long)iy * p->nx + ix] = I[c];
    }
    free(I);
  }
  (void)nthreads;
  return 0;
}

int orc_render_pixels(const orc_problem *p, const long long *pix, int npix, double *out,
                      int nthreads) {
  if (check(p)) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < npix; i++) {
    int ix = (int)(pix[i] % p->nx), iy = (int)(pix[i] / p->nx);
    march_pixel(p, NULL, ix, iy, out + (long long)i * p->nch);
  }
  (void)nthreads;
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Reverse mode of the march (hand-derived, no checkpoints: every per-sample state is kept) */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
  double *gT, *gn, *gvt, *ghlo, *ghhi;
  double *gW, *gb; /* network parameters, flat in layer order (NULL without a network) */
  double *gvphi;   /* rotation field (NULL without one) */
  /* 3-D Cartesian grid: abundance and velocity fields (gT, gn, gvt then hold the grid's
     nodes as well; ghlo, ghhi are unused) */
  double *gxco, *gvx, *gvy, *gvz;
} grads;

static void mlp_backward(const orc_mlp *m, const double xin[2], const double *gout,
                         double *gW, double *gb);

static void adjoint_pixel(const orc_problem *p, const orc_mlp *m, int ix, int iy,
                          const double *gout, double *I, grads *g) {
  double P0[3], om[3], s0, s1;
  ray_setup(p, ix, iy, P0, om);
  double conv = unit_conv(p);
  int N = p->n_samples, C = p->nch;
  if (!chord(p, P0, om, &s0, &s1)) {
    for (int c = 0; c < C; c++) I[c] = p->I0;
    return;
  }
  double ds = (s1 - s0) / N, ds_cm = ds * AU_CM;
  double hnu = H_PLANCK * p->nu0_hz / (4.0 * M_PI);
  pt *st = (pt *)malloc(sizeof(pt) * N);
  double *phi = (double *)malloc(sizeof(double) * N * C);
  double *xarg = (double *)malloc(sizeof(double) * N * C);
  double *dtau = (double *)malloc(sizeof(double) * N * C);
  double *Tr = (double *)malloc(sizeof(double) * (N + 1) * C); /* Tr[k][c] before sample k */
  double *Ic = (double *)calloc(C, sizeof(double));
  for (int c = 0; c < C; c++) Tr[c] = 1.0;
  /* forward, keeping every state */
  for (int k = 0; k < N; k++) {
    double s = s0 + (k + 0.5) * ds;
    double P[3] = {P0[0] + s * om[0], P0[1] + s * om[1], P0[2] + s * om[2]};
    eval_point(p, m, P, om, &st[k]);
    for (int c = 0; c < C; c++) {
      double tr = Tr[k * C + c];
      phi[k * C + c] = 0.0;
      dtau[k * C + c] = 0.0;
      if (st[k].gas) {
        phi[k * C + c] = profile(p, &st[k], p->v_kms[c], &xarg[k * C + c]);
        dtau[k * C + c] = hnu * st[k].D * phi[k * C + c] * ds_cm;
      }
      double dt = dtau[k * C + c];
      if (dt > 0.0) {
        Ic[c] += tr * st[k].S * (-expm1(-dt));
        Tr[(k + 1) * C + c] = tr * exp(-dt);
      } else {
        Tr[(k + 1) * C + c] = tr;
      }
    }
  }
  for (int c = 0; c < C; c++) I[c] = Ic[c] * conv + p->I0 * Tr[N * C + c];

  /* reverse */
  double B = rot_B(p);
  int Ju = p->J_u, Jl = p->J_u - 1;
  double Eu = H_PLANCK * B * Ju * (Ju + 1.0), El = H_PLANCK * B * Jl * (Jl + 1.0);
  double Bul = p->A_ul * C_LIGHT * C_LIGHT / (2.0 * H_PLANCK * pow(p->nu0_hz, 3));
  double Blu = (2.0 * Ju + 1.0) / (2.0 * Jl + 1.0) * Bul;
  double mco = p->m_co_amu * AMU_G, mmol = p->m_mol_amu * AMU_G;
  double *gI = (double *)malloc(sizeof(double) * C);
  double *gTr = (double *)malloc(sizeof(double) * C);
  for (int c = 0; c < C; c++) {
    gI[c] = gout[c] * conv;   /* dL/d(sum in cgs) */
    gTr[c] = gout[c] * p->I0; /* dL/dTr_N through the background term */
  }
  for (int k = N - 1; k >= 0; k--) {
    const pt *q = &st[k];
    double gS = 0.0, gD = 0.0, galpha = 0.0, gvlos = 0.0;
    for (int c = 0; c < C; c++) {
      double tr = Tr[k * C + c], dt = dtau[k * C + c];
      if (!(dt > 0.0)) continue; /* this step was the identity */
      double e = exp(-dt), em = -expm1(-dt);
      /* step: I += tr S em ; Tr' = tr e */
      double g_dtau = gI[c] * tr * q->S * e - gTr[c] * tr * e;
      gS += gI[c] * tr * em;
      gTr[c] = gI[c] * q->S * em + gTr[c] * e;
      /* dtau = (h nu0/4pi) D phi ds */
      double g_beta = g_dtau * ds_cm;
      gD += g_beta * hnu * phi[k * C + c];
      double g_phi = g_beta * hnu * q->D;
      /* phi = c/(nu0 alpha sqrt(pi)) exp(-x^2), x = Q/alpha: dphi/dalpha = phi (2x^2-1)/alpha */
      double xx = xarg[k * C + c];
      galpha += g_phi * phi[k * C + c] * (2.0 * xx * xx - 1.0) / q->alpha;
      /* x = (v_los - v_c) / alpha (cm/s): dphi/dv_los = -2 x phi / alpha */
      gvlos += g_phi * phi[k * C + c] * (-2.0 * xx) / q->alpha;
    }
    if (!q->gas) continue;
    /* D = n_CO Du with Du = f_l B_lu - f_u B_ul, and S = A_ul n_u / D = A_ul f_u / Du: the
       source does not depend on n_CO (it cancels), so dL/dn_CO = gD Du, and through
       f_J = g_J exp(-E_J/kT)/Z(T)
         dS/dT = A_ul B_lu (f_l f_u' - f_u f_l') / Du^2,  dD/dT = n_CO (B_lu f_l' - B_ul f_u')
       (written without dividing by D, which underflows where n_CO does) */
    double kT2 = K_BOLTZ * q->T * q->T;
    double Em = mean_energy(q->T, B);
    double dfu = q->fu * (Eu - Em) / kT2, dfl = q->fl * (El - Em) / kT2;
    double Du = q->fl * Blu - q->fu * Bul;
    double gnco = gD * Du;
    double dSdT = p->A_ul * Blu * (q->fl * dfu - q->fu * dfl) / (Du * Du);
    double gT = gS * dSdT + gD * q->nco * (Blu * dfl - Bul * dfu);
    /* alpha */
    double dadT, dadvt;
    if (p->vturb_mach) {
      dadT = (K_BOLTZ / mco + q->vt * q->vt * K_BOLTZ / mmol) / q->alpha;
      dadvt = q->vt * 2.0 * K_BOLTZ * q->T / mmol / q->alpha;
    } else {
      dadT = (K_BOLTZ / mco) / q->alpha;
      dadvt = 1e5 * (q->vt * 1e5) / q->alpha;
    }
    gT += galpha * dadT;
    double gvt = galpha * dadvt;
    /* n_CO = X n */
    double gX = gnco * q->n, gn = gnco * q->X;
    if (p->g3 || p->gs) {
      /* 3-D grids: every field is interpolated trilinearly, X is a field of its own and
         v_los is linear in the three velocity fields (d v_los / d field = dv3); the weight of
         corner (dx, dy, dz) is the product of f or 1 - f along each axis. Cartesian nodes are
         [z][y][x]; spherical ones [phi][theta][r], the azimuth periodic */
      for (int c8 = 0; c8 < 8; c8++) {
        int dx = c8 & 1, dy = (c8 >> 1) & 1, dz = c8 >> 2;
        double w = (dx ? q->f3[0] : 1.0 - q->f3[0]) * (dy ? q->f3[1] : 1.0 - q->f3[1]) *
                   (dz ? q->f3[2] : 1.0 - q->f3[2]);
        long long id;
        if (p->g3)
          id = ((long long)(q->i3[2] + dz) * p->g3->ny + (q->i3[1] + dy)) * p->g3->nx +
               (q->i3[0] + dx);
        else
          id = ((long long)(dz ? q->k1 : q->i3[2]) * p->gs->nth + (q->i3[1] + dy)) * p->gs->nr +
               (q->i3[0] + dx);
        g->gT[id] += gT * w;
        g->gn[id] += gn * w;
        g->gvt[id] += gvt * w;
        g->gxco[id] += gX * w;
        g->gvx[id] += gvlos * q->dv3[0] * w;
        g->gvy[id] += gvlos * q->dv3[1] * w;
        g->gvz[id] += gvlos * q->dv3[2] * w;
      }
      continue;
    }
    double ghlo = 0.0, ghhi = 0.0;
    if (p->edge_w > 0) {
      ghlo = gX * p->x_co * q->sb * q->sa * (1.0 - q->sa) * (-1.0 / p->edge_w);
      ghhi = gX * p->x_co * q->sa * q->sb * (1.0 - q->sb) * (1.0 / p->edge_w);
    }
    /* Neural field: T = T_grid exp(o0), n = n_grid exp(o1), h = h_grid + h_scale o2,3; the
       gradients above are with respect to the modulated values. */
    if (m) {
      double go[64] = {0};
      go[0] = gT * q->T;
      go[1] = gn * q->n;
      go[2] = ghlo * m->h_scale;
      go[3] = ghhi * m->h_scale;
      mlp_backward(m, q->xin, go, g->gW, g->gb);
    }
    gT *= q->mT;
    gn *= q->mn;
    /* bilinear scatter to the nodes */
    int nr = p->nr, i0 = q->i0, j0 = q->j0;
    double fr = q->fr, fz = q->fz;
    int idx[4] = {j0 * nr + i0, j0 * nr + i0 + 1, (j0 + 1) * nr + i0, (j0 + 1) * nr + i0 + 1};
    double wt[4] = {(1 - fr) * (1 - fz), fr * (1 - fz), (1 - fr) * fz, fr * fz};
    for (int a = 0; a < 4; a++) {
      g->gT[idx[a]] += gT * wt[a];
      g->gn[idx[a]] += gn * wt[a];
      g->gvt[idx[a]] += gvt * wt[a];
    }
    g->ghlo[i0] += ghlo * (1 - fr);
    g->ghlo[i0 + 1] += ghlo * fr;
    g->ghhi[i0] += ghhi * (1 - fr);
    g->ghhi[i0 + 1] += ghhi * fr;
    if (g->gvphi)
      for (int a = 0; a < 4; a++) g->gvphi[idx[a]] += gvlos * q->dvlos_dvphi * wt[a];
  }
  free(gI);
  free(gTr);
  free(st);
  free(phi);
  free(xarg);
  free(dtau);
  free(Tr);
  free(Ic);
}

static int mlp_check(const orc_mlp *m);

static long long mlp_nw(const orc_mlp *m) {
  long long n = 0;
  for (int l = 0; l < m->n_layers; l++) n += (long long)m->dims[l + 1] * m->dims[l];
  return n;
}

static long long mlp_nb(const orc_mlp *m) {
  long long n = 0;
  for (int l = 0; l < m->n_layers; l++) n += m->dims[l + 1];
  return n;
}

static int render_adjoint_impl(const orc_problem *p, const orc_mlp *m, const double *dL_dcube,
                               double *cube, double *dT, double *dn, double *dvt, double *dh_lo,
                               double *dh_hi, double *dW, double *db, double *dvphi,
                               int nthreads) {
  if (check(p) || !dL_dcube || p->g3 || p->gs) return -1; /* axisymmetric grid only */
  if (m && (mlp_check(m) || m->dims[m->n_layers] < 4 || m->dims[m->n_layers] > 64)) return -1;
  int G = p->nr * p->nz;
  long long npix = (long long)p->nx * p->ny;
  long long nw = m ? mlp_nw(m) : 0, nb = m ? mlp_nb(m) : 0;
  memset(dT, 0, sizeof(double) * G);
  memset(dn, 0, sizeof(double) * G);
  memset(dvt, 0, sizeof(double) * G);
  memset(dh_lo, 0, sizeof(double) * p->nr);
  memset(dh_hi, 0, sizeof(double) * p->nr);
  if (dvphi) memset(dvphi, 0, sizeof(double) * G);
  if (m) {
    memset(dW, 0, sizeof(double) * nw);
    memset(db, 0, sizeof(double) * nb);
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    grads g;
    g.gT = (double *)calloc(G, sizeof(double));
    g.gn = (double *)calloc(G, sizeof(double));
    g.gvt = (double *)calloc(G, sizeof(double));
    g.ghlo = (double *)calloc(p->nr, sizeof(double));
    g.ghhi = (double *)calloc(p->nr, sizeof(double));
    g.gW = m ? (double *)calloc(nw, sizeof(double)) : NULL;
    g.gb = m ? (double *)calloc(nb, sizeof(double)) : NULL;
    g.gvphi = dvphi ? (double *)calloc(G, sizeof(double)) : NULL;
    double *gout = (double *)malloc(sizeof(double) * (p->nch > 0 ? p->nch : 1));
    double *I = (double *)malloc(sizeof(double) * (p->nch > 0 ? p->nch : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int iy = 0; iy < p->ny; iy++) {
      for (int ix = 0; ix < p->nx; ix++) {
        long long pix = (long long)iy * p->nx + ix;
        for (int c = 0; c < p->nch; c++) gout[c] = dL_dcube[c * npix + pix];
        adjoint_pixel(p, m, ix, iy, gout, I, &g);
        if (cube)
          for (int c = 0; c < p->nch; c++) cube[c * npix + pix] = I[c];
      }
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    {
      for (int a = 0; a < G; a++) {
        dT[a] += g.gT[a];
        dn[a] += g.gn[a];
        dvt[a] += g.gvt[a];
      }
      for (int a = 0; a < p->nr; a++) {
        dh_lo[a] += g.ghlo[a];
        dh_hi[a] += g.ghhi[a];
      }
      if (dvphi)
        for (int a = 0; a < G; a++) dvphi[a] += g.gvphi[a];
      for (long long a = 0; a < nw; a++) dW[a] += g.gW[a];
      for (long long a = 0; a < nb; a++) db[a] += g.gb[a];
    }
    free(g.gT);
    free(g.gn);
    free(g.gvt);
    free(g.ghlo);
    free(g.ghhi);
    free(g.gW);
    free(g.gb);
    free(g.gvphi);
    free(gout);
    free(I);
  }
  (void)nthreads;
  return 0;
}

int orc_render_adjoint(const orc_problem *p, const double *dL_dcube, double *cube,
                       double *dT, double *dn, double *dvt, double *dh_lo, double *dh_hi,
                       int nthreads) {
  return render_adjoint_impl(p, NULL, dL_dcube, cube, dT, dn, dvt, dh_lo, dh_hi, NULL, NULL,
                             NULL, nthreads);
}

int orc_render_adjoint_vphi(const orc_problem *p, const double *dL_dcube, double *cube,
                            double *dT, double *dn, double *dvt, double *dh_lo, double *dh_hi,
                            double *dvphi, int nthreads) {
  if (!p || !p->vphi || !dvphi) return -1;
  return render_adjoint_impl(p, NULL, dL_dcube, cube, dT, dn, dvt, dh_lo, dh_hi, NULL, NULL,
                             dvphi, nthreads);
}

int orc_render_adjoint3(const orc_problem *p, const double *dL_dcube, double *cube, double *dT,
                        double *dn, double *dvt, double *dxco, double *dvx, double *dvy,
                        double *dvz, int nthreads) {
  if (!p || !p->g3 == !p->gs || check(p) || !dL_dcube) return -1;
  long long G = p->g3 ? (long long)p->g3->nx * p->g3->ny * p->g3->nz
                      : (long long)p->gs->nr * p->gs->nth * p->gs->nph;
  long long npix = (long long)p->nx * p->ny;
  double *out[7] = {dT, dn, dvt, dxco, dvx, dvy, dvz};
  for (int a = 0; a < 7; a++) memset(out[a], 0, sizeof(double) * G);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    grads g;
    memset(&g, 0, sizeof(g));
    double *acc[7];
    for (int a = 0; a < 7; a++) acc[a] = (double *)calloc(G, sizeof(double));
    g.gT = acc[0];
    g.gn = acc[1];
    g.gvt = acc[2];
    g.gxco = acc[3];
    g.gvx = acc[4];
    g.gvy = acc[5];
    g.gvz = acc[6];
    double *gout = (double *)malloc(sizeof(double) * (p->nch > 0 ? p->nch : 1));
    double *I = (double *)malloc(sizeof(double) * (p->nch > 0 ? p->nch : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int iy = 0; iy < p->ny; iy++) {
      for (int ix = 0; ix < p->nx; ix++) {
        long long pix = (long long)iy * p->nx + ix;
        for (int c = 0; c < p->nch; c++) gout[c] = dL_dcube[c * npix + pix];
        adjoint_pixel(p, NULL, ix, iy, gout, I, &g);
        if (cube)
          for (int c = 0; c < p->nch; c++) cube[c * npix + pix] = I[c];
      }
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    {
      for (int a = 0; a < 7; a++)
        for (long long i = 0; i < G; i++) out[a][i] += acc[a][i];
    }
    for (int a = 0; a < 7; a++) free(acc[a]);
    free(gout);
    free(I);
  }
  (void)nthreads;
  return 0;
}

int orc_render_mlp_adjoint(const orc_problem *p, const orc_mlp *m, const double *dL_dcube,
                           double *cube, double *dT, double *dn, double *dvt, double *dh_lo,
                           double *dh_hi, double *dW, double *db, int nthreads) {
  if (!m || !dW || !db) return -1;
  return render_adjoint_impl(p, m, dL_dcube, cube, dT, dn, dvt, dh_lo, dh_hi, dW, db, NULL,
                             nthreads);
}

/* ---------------------------------------------------------------------------------------- */
/* Neural field (the symmetric MLP T(r,|z|) = MLP_w(gamma(r,|z|)) of the neural-temperature */
/* section, with Fourier-feature encoding gamma and SiLU hidden activations)               */
/* ---------------------------------------------------------------------------------------- */

static void mlp_forward(const orc_mlp *m, const double xin[2], double *out) {
  double buf1[ORC_MLP_MAXW], buf2[ORC_MLP_MAXW];
  double *h = buf1, *h2 = buf2;
  /* gamma(x): [sin(2 pi B x), cos(2 pi B x)] */
  for (int f = 0; f < m->n_freq; f++) {
    double a = 2.0 * M_PI * (m->B[2 * f] * xin[0] + m->B[2 * f + 1] * xin[1]);
    h[f] = sin(a);
    h[m->n_freq + f] = cos(a);
  }
  for (int l = 0; l < m->n_layers; l++) {
    int din = m->dims[l], dout = m->dims[l + 1];
    for (int o = 0; o < dout; o++) {
      double acc = m->b[l][o];
      for (int i = 0; i < din; i++) acc += m->W[l][(long long)o * din + i] * h[i];
      /* SiLU on hidden layers, identity on the output layer */
      h2[o] = (l < m->n_layers - 1) ? acc / (1.0 + exp(-acc)) : acc;
    }
    double *t = h;
    h = h2;
    h2 = t;
  }
  for (int o = 0; o < m->dims[m->n_layers]; o++) out[o] = h[o];
}

/* Reverse mode of mlp_forward at input xin for output gradient gout: accumulates
   dL/dW (flat, layer after layer, each [dims[l+1]][dims[l]]) and dL/db. SiLU'(z) =
   s (1 + z (1 - s)) with s the logistic function of z. */
static void mlp_backward(const orc_mlp *m, const double xin[2], const double *gout,
                         double *gW, double *gb) {
  int L = m->n_layers;
  double *act = (double *)malloc(sizeof(double) * (L + 1) * ORC_MLP_MAXW); /* a_0 .. a_L */
  double *pre = (double *)malloc(sizeof(double) * (L + 1) * ORC_MLP_MAXW); /* z_1 .. z_L */
  double *d = (double *)malloc(sizeof(double) * ORC_MLP_MAXW);
  double *d2 = (double *)malloc(sizeof(double) * ORC_MLP_MAXW);
  for (int f = 0; f < m->n_freq; f++) {
    double a = 2.0 * M_PI * (m->B[2 * f] * xin[0] + m->B[2 * f + 1] * xin[1]);
    act[f] = sin(a);
    act[m->n_freq + f] = cos(a);
  }
  for (int l = 0; l < L; l++) {
    int din = m->dims[l], dout = m->dims[l + 1];
    const double *a = act + (long long)l * ORC_MLP_MAXW;
    double *z = pre + (long long)(l + 1) * ORC_MLP_MAXW;
    double *an = act + (long long)(l + 1) * ORC_MLP_MAXW;
    for (int o = 0; o < dout; o++) {
      double acc = m->b[l][o];
      for (int i = 0; i < din; i++) acc += m->W[l][(long long)o * din + i] * a[i];
      z[o] = acc;
      an[o] = (l < L - 1) ? acc / (1.0 + exp(-acc)) : acc;
    }
  }
  /* offsets of each layer in the flat gradient arrays */
  long long offW = 0, offb = 0;
  for (int l = 0; l < L - 1; l++) {
    offW += (long long)m->dims[l + 1] * m->dims[l];
    offb += m->dims[l + 1];
  }
  for (int o = 0; o < m->dims[L]; o++) d[o] = gout[o]; /* dL/da_L (identity output layer) */
  for (int l = L - 1; l >= 0; l--) {
    int din = m->dims[l], dout = m->dims[l + 1];
    const double *a = act + (long long)l * ORC_MLP_MAXW;
    const double *z = pre + (long long)(l + 1) * ORC_MLP_MAXW;
    /* dL/dz_{l+1} */
    if (l < L - 1)
      for (int o = 0; o < dout; o++) {
        double sg = 1.0 / (1.0 + exp(-z[o]));
        d[o] *= sg * (1.0 + z[o] * (1.0 - sg));
      }
    for (int o = 0; o < dout; o++) {
      gb[offb + o] += d[o];
      for (int i = 0; i < din; i++) gW[offW + (long long)o * din + i] += d[o] * a[i];
    }
    if (l > 0) {
      for (int i = 0; i < din; i++) {
        double acc = 0.0;
        for (int o = 0; o < dout; o++) acc += m->W[l][(long long)o * din + i] * d[o];
        d2[i] = acc;
      }
      for (int i = 0; i < din; i++) d[i] = d2[i];
      offW -= (long long)m->dims[l] * m->dims[l - 1];
      offb -= m->dims[l];
    }
  }
  free(act);
  free(pre);
  free(d);
  free(d2);
}

static int mlp_check(const orc_mlp *m) {
  if (!m || m->n_layers < 1 || m->dims[0] != 2 * m->n_freq) return -1;
  for (int l = 0; l <= m->n_layers; l++)
    if (m->dims[l] < 1 || m->dims[l] > ORC_MLP_MAXW) return -1;
  return 0;
}

int orc_mlp_eval(const orc_mlp *m, const double *x, int npts, double *out) {
  if (mlp_check(m)) return -1;
  int no = m->dims[m->n_layers];
  for (int i = 0; i < npts; i++) {
    double o[64];
    if (no > 64) return -1;
    mlp_forward(m, x + 2 * i, o);
    for (int a = 0; a < no; a++) out[(long long)i * no + a] = o[a];
  }
  return 0;
}

int orc_mlp_grad(const orc_mlp *m, const double *x, const double *gout, int npts, double *dW,
                 double *db) {
  if (mlp_check(m) || m->dims[m->n_layers] > 64) return -1;
  int no = m->dims[m->n_layers];
  memset(dW, 0, sizeof(double) * mlp_nw(m));
  memset(db, 0, sizeof(double) * mlp_nb(m));
  for (int i = 0; i < npts; i++) mlp_backward(m, x + 2 * i, gout + (long long)i * no, dW, db);
  return 0;
}

int orc_render_mlp(const orc_problem *p, const orc_mlp *m, const long long *pix, int npix,
                   double *out, int nthreads) {
  if (check(p) || mlp_check(m) || m->dims[m->n_layers] < 4 || p->g3 || p->gs) return -1;
  long long np = pix ? npix : (long long)p->nx * p->ny;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (long long i = 0; i < np; i++) {
    long long q = pix ? pix[i] : i;
    int ix = (int)(q % p->nx), iy = (int)(q / p->nx);
    double *I = (double *)malloc(sizeof(double) * (p->nch > 0 ? p->nch : 1));
    march_pixel(p, m, ix, iy, I);
    for (int c = 0; c < p->nch; c++) {
      if (pix)
        out[i * p->nch + c] = I[c];
      else
        out[(long long)c * p->nx * p->ny + q] = I[c];
    }
    free(I);
  }
  (void)nthreads;
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Physics-constrained field chain (see rt_oracle.h): hydrostatic density from a temperature
 * grid, H2 column above each node, CO-layer surfaces. One radius column at a time, nodes in
 * order; every integral is the trapezoid rule on the grid nodes.
 * ------------------------------------------------------------------------------------------ */
int orc_field_chain(const orc_problem *p, const orc_chain *c, const double *T, double *n_h2,
                    double *N_h2, double *h_lo, double *h_hi) {
  if (!p || !c || !T || !n_h2 || !h_lo || !h_hi || p->nr < 2 || p->nz < 2) return -1;
  const int nr = p->nr, nz = p->nz;
  const double GM = GM_SUN * p->mstar_msun;          /* cm^3 s^-2 */
  const double m_mol = p->m_mol_amu * AMU_G;         /* g */
  double *z = (double *)malloc(sizeof(double) * nz); /* node heights [cm] */
  double *lnrho = (double *)malloc(sizeof(double) * nz);
  double *N = (double *)malloc(sizeof(double) * nz);
  if (!z || !lnrho || !N) {
    free(z);
    free(lnrho);
    free(N);
    return -1;
  }
  for (int i = 0; i < nr; i++) {
    double r_au = p->r_log ? p->r_in_au * pow(p->r_out_au / p->r_in_au, (double)i / (nr - 1))
                           : p->r_in_au + (p->r_out_au - p->r_in_au) * i / (nr - 1);
    double r = r_au * AU_CM;
    for (int j = 0; j < nz; j++) z[j] = p->zr_max * j / (nz - 1) * r;
    /* Eq. gas_density_temp: the gravity term by the trapezoid rule, the temperature term
       integrates to -ln(T_j / T_0) */
    double grav_prev = 0.0, I = 0.0;
    for (int j = 0; j < nz; j++) {
      double Tj = T[(long long)j * nr + i];
      double d3 = pow(r * r + z[j] * z[j], 1.5);
      double grav = GM * z[j] / d3 * m_mol / (K_BOLTZ * Tj);
      if (j > 0) I += 0.5 * (z[j] - z[j - 1]) * (grav_prev + grav);
      grav_prev = grav;
      lnrho[j] = -I - log(Tj / T[i]);
    }
    /* normalisation: 2 int_0^{z_max} rho dz = Sigma(r) */
    double x = r_au / c->r_c_au;
    double sigma = c->sigma0_gcm2 * pow(x, -c->gamma) * exp(-pow(x, 2.0 - c->gamma));
    double S = 0.0;
    for (int j = 1; j < nz; j++) S += 0.5 * (z[j] - z[j - 1]) * (exp(lnrho[j - 1]) + exp(lnrho[j]));
    for (int j = 0; j < nz; j++)
      n_h2[(long long)j * nr + i] = sigma / (2.0 * S) * exp(lnrho[j]) / m_mol;
    /* Eq. column_density: N(z_j) = int_{z_j}^{z_max} n dz */
    N[nz - 1] = 0.0;
    for (int j = nz - 2; j >= 0; j--)
      N[j] = N[j + 1] + 0.5 * (z[j + 1] - z[j]) *
                            (n_h2[(long long)j * nr + i] + n_h2[(long long)(j + 1) * nr + i]);
    if (N_h2)
      for (int j = 0; j < nz; j++) N_h2[(long long)j * nr + i] = N[j];
    /* Eq. co_layer as two surfaces (w = z/r) */
    double dw = p->zr_max / (nz - 1);
    double lo = p->zr_max;
    if (T[i] > c->T_freeze) {
      lo = 0.0;
    } else {
      for (int j = 1; j < nz; j++) {
        double Ta = T[(long long)(j - 1) * nr + i], Tb = T[(long long)j * nr + i];
        if (Tb > c->T_freeze) {
          lo = dw * ((j - 1) + (c->T_freeze - Ta) / (Tb - Ta));
          break;
        }
      }
    }
    double hi = 0.0;
    for (int j = nz - 2; j >= 0; j--) {
      if (0.706 * N[j] > c->N_dissoc_cm2) {
        double Na = 0.706 * N[j], Nb = 0.706 * N[j + 1];
        hi = dw * (j + (Na - c->N_dissoc_cm2) / (Na - Nb));
        break;
      }
    }
    h_lo[i] = lo;
    h_hi[i] = hi;
  }
  free(z);
  free(lnrho);
  free(N);
  return 0;
}

/* Reverse mode of orc_field_chain (see rt_oracle.h): per column, the forward quantities
   again, then their adjoints in the reverse order of the forward steps. */
int orc_field_chain_adjoint(const orc_problem *p, const orc_chain *c, const double *T,
                            const double *g_n, const double *g_lo, const double *g_hi,
                            double *g_T) {
  if (!p || !c || !T || !g_T || p->nr < 2 || p->nz < 2) return -1;
  const int nr = p->nr, nz = p->nz;
  const double GM = GM_SUN * p->mstar_msun;
  const double m_mol = p->m_mol_amu * AMU_G;
  double *buf = (double *)malloc(sizeof(double) * 8 * nz);
  if (!buf) return -1;
  double *z = buf, *grav = buf + nz, *e = buf + 2 * nz, *n = buf + 3 * nz, *N = buf + 4 * nz;
  double *gN = buf + 5 * nz, *gn = buf + 6 * nz, *gI = buf + 7 * nz;
  for (int i = 0; i < nr; i++) {
    const double r_au = p->r_log ? p->r_in_au * pow(p->r_out_au / p->r_in_au, (double)i / (nr - 1))
                                 : p->r_in_au + (p->r_out_au - p->r_in_au) * i / (nr - 1);
    const double r = r_au * AU_CM;
    const double *Tc = T + i; /* T of node j: Tc[j * nr] */
    /* forward: gravity term, its trapezoid integral I, rho up to the normalisation (e),
       the normalisation S, n and the column N */
    double I = 0.0;
    for (int j = 0; j < nz; j++) {
      z[j] = p->zr_max * j / (nz - 1) * r;
      grav[j] = GM * z[j] / pow(r * r + z[j] * z[j], 1.5) * m_mol / (K_BOLTZ * Tc[(long long)j * nr]);
      if (j > 0) I += 0.5 * (z[j] - z[j - 1]) * (grav[j - 1] + grav[j]);
      e[j] = exp(-I - log(Tc[(long long)j * nr] / Tc[0]));
    }
    const double x = r_au / c->r_c_au;
    const double sigma = c->sigma0_gcm2 * pow(x, -c->gamma) * exp(-pow(x, 2.0 - c->gamma));
    double S = 0.0;
    for (int j = 1; j < nz; j++) S += 0.5 * (z[j] - z[j - 1]) * (e[j - 1] + e[j]);
    const double Cn = sigma / (2.0 * S) / m_mol; /* n_j = Cn e_j */
    for (int j = 0; j < nz; j++) n[j] = Cn * e[j];
    N[nz - 1] = 0.0;
    for (int j = nz - 2; j >= 0; j--) N[j] = N[j + 1] + 0.5 * (z[j + 1] - z[j]) * (n[j] + n[j + 1]);
    for (int j = 0; j < nz; j++) {
      g_T[(long long)j * nr + i] = 0.0;
      gN[j] = 0.0;
      gn[j] = g_n ? g_n[(long long)j * nr + i] : 0.0;
    }
    const double dw = p->zr_max / (nz - 1);
    /* h_hi = dw (j + (Na - Nd) / (Na - Nb)) in the highest cell [j, j+1] with 0.706 N_j > Nd */
    if (g_hi && g_hi[i] != 0.0) {
      for (int j = nz - 2; j >= 0; j--) {
        if (0.706 * N[j] > c->N_dissoc_cm2) {
          const double Na = 0.706 * N[j], Nb = 0.706 * N[j + 1], Nd = c->N_dissoc_cm2;
          const double q = (Na - Nb) * (Na - Nb);
          gN[j] += g_hi[i] * dw * (Nd - Nb) / q * 0.706;
          gN[j + 1] += g_hi[i] * dw * (Na - Nd) / q * 0.706;
          break;
        }
      }
    }
    /* N_j = sum_{k >= j} (dz/2)(n_k + n_{k+1}): dL/dn_k from every N_j with j <= k */
    double P = 0.0; /* sum_{j <= k} gN_j */
    for (int k = 0; k < nz; k++) {
      const double Pprev = P;
      P += gN[k];
      if (k <= nz - 2) gn[k] += 0.5 * (z[k + 1] - z[k]) * P;
      if (k >= 1) gn[k] += 0.5 * (z[k] - z[k - 1]) * Pprev;
    }
    /* n_j = Cn e_j, Cn = sigma / (2 S m): dL/de_k = Cn gn_k - (Cn / S) w_k sum_j gn_j e_j,
       w_k the trapezoid weight of node k in S */
    double ge_dot = 0.0;
    for (int j = 0; j < nz; j++) ge_dot += gn[j] * e[j];
    double gT0 = 0.0;
    for (int k = 0; k < nz; k++) {
      const double wk = (k > 0 ? 0.5 * (z[k] - z[k - 1]) : 0.0) + (k < nz - 1 ? 0.5 * (z[k + 1] - z[k]) : 0.0);
      const double ge = Cn * gn[k] - Cn / S * wk * ge_dot;
      /* e_k = exp(lnrho_k), lnrho_k = -I_k - ln T_k + ln T_0 */
      const double glr = ge * e[k];
      gI[k] = -glr;
      g_T[(long long)k * nr + i] += -glr / Tc[(long long)k * nr];
      gT0 += glr / Tc[0];
    }
    g_T[i] += gT0;
    /* I_j = sum_{m=1}^{j} (dz_m / 2)(grav_{m-1} + grav_m); grav_m = a_m / T_m */
    double Q = 0.0; /* sum_{j >= m + 1} gI_j, accumulated from the top */
    for (int m = nz - 1; m >= 0; m--) {
      double gg = 0.0;
      if (m + 1 <= nz - 1) gg += 0.5 * (z[m + 1] - z[m]) * Q;        /* as grav_{(m+1)-1} */
      if (m >= 1) gg += 0.5 * (z[m] - z[m - 1]) * (Q + gI[m]);      /* as grav_m, j >= m */
      Q += gI[m];
      g_T[(long long)m * nr + i] += -gg * grav[m] / Tc[(long long)m * nr];
    }
    /* h_lo = dw ((j - 1) + (Tf - Ta) / (Tb - Ta)) in the lowest cell [j-1, j] with Tb > Tf */
    if (g_lo && g_lo[i] != 0.0 && !(Tc[0] > c->T_freeze)) {
      for (int j = 1; j < nz; j++) {
        const double Ta = Tc[(long long)(j - 1) * nr], Tb = Tc[(long long)j * nr];
        if (Tb > c->T_freeze) {
          const double q = (Tb - Ta) * (Tb - Ta), Tf = c->T_freeze;
          g_T[(long long)(j - 1) * nr + i] += g_lo[i] * dw * (Tf - Tb) / q;
          g_T[(long long)j * nr + i] += -g_lo[i] * dw * (Tf - Ta) / q;
          break;
        }
      }
    }
  }
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Pressure-corrected rotation (see rt_oracle.h), node by node.
 * ------------------------------------------------------------------------------------------ */
static double node_r_au(const orc_problem *p, int i) {
  return p->r_log ? p->r_in_au * pow(p->r_out_au / p->r_in_au, (double)i / (p->nr - 1))
                  : p->r_in_au + (p->r_out_au - p->r_in_au) * i / (p->nr - 1);
}

/* derivative of f along an axis of n uniformly spaced nodes (spacing h) at node k, from
   the values f(k') = F[k' * stride] */
static double axis_diff(const double *F, long long stride, int n, int k, double h) {
  if (n == 2) return (F[stride] - F[0]) / h;
  if (k == 0) return (-3.0 * F[0] + 4.0 * F[stride] - F[2 * stride]) / (2.0 * h);
  if (k == n - 1)
    return (3.0 * F[k * stride] - 4.0 * F[(k - 1) * stride] + F[(k - 2) * stride]) / (2.0 * h);
  return (F[(k + 1) * stride] - F[(k - 1) * stride]) / (2.0 * h);
}

/* adds g c_l to G[l stride] for the coefficients c_l of axis_diff at node k */
static void axis_diff_adjoint(double *G, long long stride, int n, int k, double h, double g) {
  if (n == 2) {
    G[0] += -g / h;
    G[stride] += g / h;
  } else if (k == 0) {
    G[0] += -3.0 * g / (2.0 * h);
    G[stride] += 4.0 * g / (2.0 * h);
    G[2 * stride] += -g / (2.0 * h);
  } else if (k == n - 1) {
    G[k * stride] += 3.0 * g / (2.0 * h);
    G[(k - 1) * stride] += -4.0 * g / (2.0 * h);
    G[(k - 2) * stride] += g / (2.0 * h);
  } else {
    G[(k + 1) * stride] += g / (2.0 * h);
    G[(k - 1) * stride] += -g / (2.0 * h);
  }
}

/* Reverse mode of orc_pressure_vphi (see rt_oracle.h). */
int orc_pressure_vphi_adjoint(const orc_problem *p, const double *n_h2, const double *T,
                              const double *g_v, double *g_n, double *g_T) {
  if (!p || !n_h2 || !T || !g_v || !g_n || !g_T || p->nr < 2 || p->nz < 2) return -1;
  const int nr = p->nr, nz = p->nz;
  const long long G = (long long)nr * nz;
  double *P = (double *)malloc(sizeof(double) * G);
  double *gP = (double *)calloc(G, sizeof(double));
  if (!P || !gP) {
    free(P);
    free(gP);
    return -1;
  }
  for (long long k = 0; k < G; k++) {
    P[k] = n_h2[k] * K_BOLTZ * T[k];
    g_n[k] = 0.0;
    g_T[k] = 0.0;
  }
  const double hu = p->r_log ? log(p->r_out_au / p->r_in_au) / (nr - 1)
                             : (p->r_out_au - p->r_in_au) * AU_CM / (nr - 1);
  const double hw = p->zr_max / (nz - 1);
  const double GM = GM_SUN * p->mstar_msun, m = p->m_mol_amu * AMU_G;
  for (int j = 0; j < nz; j++) {
    const double w = hw * j;
    for (int i = 0; i < nr; i++) {
      const long long k = (long long)j * nr + i;
      if (!(n_h2[k] > 0.0)) continue; /* the Keplerian term alone: no dependence on n, T */
      const double r = node_r_au(p, i) * AU_CM, z = w * r;
      const double kep = GM * r * r / pow(r * r + z * z, 1.5);
      const double dPu = axis_diff(P + (long long)j * nr, 1, nr, i, hu);
      const double dPw = axis_diff(P + i, nr, nz, j, hw);
      const double dudr = p->r_log ? 1.0 / r : 1.0;
      const double dPdr = dudr * dPu - (w / r) * dPw;
      const double v2 = kep + r / (m * n_h2[k]) * dPdr;
      if (!(v2 > 0.0)) continue; /* clamped to 0: zero derivative */
      /* v [km/s] = sqrt(v2) / 1e5 */
      const double g2 = g_v[k] / (2.0 * sqrt(v2) * 1e5);
      g_n[k] += -g2 * r / (m * n_h2[k] * n_h2[k]) * dPdr;
      const double gdPdr = g2 * r / (m * n_h2[k]);
      axis_diff_adjoint(gP + (long long)j * nr, 1, nr, i, hu, gdPdr * dudr);
      axis_diff_adjoint(gP + i, nr, nz, j, hw, -gdPdr * (w / r));
    }
  }
  /* P = n k T */
  for (long long k = 0; k < G; k++) {
    g_n[k] += gP[k] * K_BOLTZ * T[k];
    g_T[k] += gP[k] * K_BOLTZ * n_h2[k];
  }
  free(P);
  free(gP);
  return 0;
}

int orc_pressure_vphi(const orc_problem *p, const double *n_h2, const double *T, double *vphi) {
  if (!p || !n_h2 || !T || !vphi || p->nr < 2 || p->nz < 2) return -1;
  const int nr = p->nr, nz = p->nz;
  double *P = (double *)malloc(sizeof(double) * (size_t)nr * nz);
  if (!P) return -1;
  for (long long k = 0; k < (long long)nr * nz; k++) P[k] = n_h2[k] * K_BOLTZ * T[k];
  const double hu = p->r_log ? log(p->r_out_au / p->r_in_au) / (nr - 1)
                             : (p->r_out_au - p->r_in_au) * AU_CM / (nr - 1);
  const double hw = p->zr_max / (nz - 1);
  const double GM = GM_SUN * p->mstar_msun, m = p->m_mol_amu * AMU_G;
  for (int j = 0; j < nz; j++) {
    const double w = hw * j;
    for (int i = 0; i < nr; i++) {
      const double r = node_r_au(p, i) * AU_CM, z = w * r;
      const double kep = GM * r * r / pow(r * r + z * z, 1.5);
      const long long k = (long long)j * nr + i;
      double v2 = kep;
      if (n_h2[k] > 0.0) {
        const double dPu = axis_diff(P + (long long)j * nr, 1, nr, i, hu);
        const double dPw = axis_diff(P + i, nr, nz, j, hw);
        const double dudr = p->r_log ? 1.0 / r : 1.0;
        const double dPdr = dudr * dPu - (w / r) * dPw;
        v2 += r / (m * n_h2[k]) * dPdr;
      }
      vphi[k] = v2 > 0.0 ? sqrt(v2) / 1e5 : 0.0;
    }
  }
  free(P);
  return 0;
}
