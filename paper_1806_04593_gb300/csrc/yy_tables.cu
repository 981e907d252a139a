// Density-independent tables of the Yin-Yang multipole solver, built once per
// grid in float64 on the GPU (§3: only the density-dependent terms change
// between solves).
//
//  k_weights        overlap surface weights w_jk (§4)
//  k_tbar           K_lm T_j^(lm), T of Eq. tlm, by Gauss-Legendre quadrature
//                   of the normalised Legendre functions
//  k_analysis_table w_jk K_lm T_j^(lm) {C_k^(m), S_k^(m)} (§2 closed forms for C, S)
//  k_synth_tables   K_lm P_l^m {cos, sin}(m phi) at the cell centre and its
//                   angular derivatives in the patch's own spherical basis
//  k_rot_points,    per degree l, the matrix D^l that expresses a harmonic
//  k_rot_accum      taken in the other patch's angles (Eqs. trafotheta /
//                   trafophi) through the own-frame harmonics of the same l
//  k_scan_coeffs    per-zone factors of the scaled radial recurrences
//                   (Eqs. rin / rout, phiin / phiout)
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "yy_internal.h"

namespace yy {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

__device__ __forceinline__ int tri(int l, int m) { return l * (l + 1) / 2 + m; }

// ---------------------------------------------------------------------------
// overlap weights
// ---------------------------------------------------------------------------
//
// In own-patch Cartesian coordinates the other patch is the set
//   |y| <= c1 r,  c1 = cos(pi/4 - delta_theta)      (its theta interval)
//   not (x > 0 and |z| < t2 x),  t2 = tan(pi/4 - delta_phi)   (its phi interval)
// since the other patch sees cos(theta') = y / r and phi' = atan2(z, -x).
// At fixed azimuth phi, with u = cos(theta), both conditions only involve u^2:
//   |y| <= c1 r         <=>  u^2 >= 1 - c1^2 / sin^2(phi)
//   |z| <  t2 x (x > 0) <=>  u^2 <  t2^2 cos^2(phi) / (1 + t2^2 cos^2(phi))
// so the point is inside iff |u| >= h(phi), h^2 the larger right-hand side.
// The solid angle of a cell column [u_hi, u_lo] inside is then the length of
// [u_hi, u_lo] outside (-h, h).

struct WeightGeom {
  double th0, ph0, dth, dph, c1, t2;
  int n_theta, n_phi;
};

__device__ __forceinline__ double other_patch_h(double phi, double c1, double t2) {
  const double s = sin(phi), c = cos(phi);
  const double s2 = s * s;
  double v = 0.0;
  if (s2 > c1 * c1) v = 1.0 - c1 * c1 / s2;
  if (c > 0.0) {
    const double tc2 = t2 * t2 * c * c;
    v = fmax(v, tc2 / (1.0 + tc2));
  }
  return sqrt(v);
}

__device__ __forceinline__ double inside_measure(double phi, double u_hi, double u_lo,
                                                 double c1, double t2) {
  const double h = other_patch_h(phi, c1, t2);
  const double cut = fmax(0.0, fmin(u_lo, h) - fmax(u_hi, -h));
  return (u_lo - u_hi) - cut;
}

__device__ __forceinline__ void push_abs_sin(double v, double lo, double hi, double *bp, int &nb) {
  if (v >= 0.0 && v <= 1.0) {
    const double a = asin(v);
    const double c[4] = {a, -a, kPi - a, a - kPi};
    for (int i = 0; i < 4; ++i)
      if (c[i] > lo && c[i] < hi) bp[nb++] = c[i];
  }
}

__device__ __forceinline__ void push_cos(double v, double lo, double hi, double *bp, int &nb) {
  if (v >= -1.0 && v <= 1.0) {
    const double a = acos(v);
    if (a > lo && a < hi) bp[nb++] = a;
    if (-a > lo && -a < hi) bp[nb++] = -a;
  }
}

// One thread per cell.  The azimuthal integral of the inside measure is
// split at every azimuth where h(phi) meets an edge |u_e|, where the two
// conditions swap, where |sin phi| = c1 (square-root branch point) and where
// cos phi = 0.  Each piece [a, b] is mapped by phi = a + (b - a)(1 - cos(pi t))/2,
// which turns square-root endpoint behaviour into an analytic integrand, and
// integrated with a 32-point Gauss-Legendre rule.
__global__ void k_weights(WeightGeom G, const double *__restrict__ gl, double *__restrict__ w) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= G.n_theta * G.n_phi) return;
  const int j = cell / G.n_phi, k = cell % G.n_phi;
  const double th_lo = G.th0 + G.dth * j, th_hi = G.th0 + G.dth * (j + 1);
  const double ph_lo = G.ph0 + G.dph * k, ph_hi = G.ph0 + G.dph * (k + 1);
  const double u_lo = cos(th_lo), u_hi = cos(th_hi);

  double bp[24];
  int nb = 0;
  bp[nb++] = ph_lo;
  push_abs_sin(G.c1, ph_lo, ph_hi, bp, nb);
  push_cos(0.0, ph_lo, ph_hi, bp, nb);
  const double th_e[2] = {th_lo, th_hi};
  for (int e = 0; e < 2; ++e) {
    const double st = sin(th_e[e]);
    if (st > 0.0) {
      push_abs_sin(G.c1 / st, ph_lo, ph_hi, bp, nb);
      push_cos(fabs(cos(th_e[e])) / st / G.t2, ph_lo, ph_hi, bp, nb);
    }
  }
  push_cos(sqrt((1.0 - G.c1 * G.c1) / (1.0 + G.c1 * G.c1 * G.t2 * G.t2)), ph_lo, ph_hi, bp, nb);
  bp[nb++] = ph_hi;
  // insertion sort (nb <= 24)
  for (int i = 1; i < nb; ++i) {
    const double v = bp[i];
    int q = i - 1;
    while (q >= 0 && bp[q] > v) {
      bp[q + 1] = bp[q];
      --q;
    }
    bp[q + 1] = v;
  }
  double area = 0.0;
  for (int p = 0; p + 1 < nb; ++p) {
    const double a = bp[p], b = bp[p + 1];
    if (!(b > a)) continue;
    double acc = 0.0;
    for (int q = 0; q < YY_GL_WEIGHT_NODES; ++q) {
      const double t = gl[q], wq = gl[YY_GL_WEIGHT_NODES + q];
      const double phi = a + (b - a) * 0.5 * (1.0 - cospi(t));
      const double jac = (b - a) * 0.5 * kPi * sinpi(t);
      acc += wq * jac * inside_measure(phi, u_hi, u_lo, G.c1, G.t2);
    }
    area += acc;
  }
  const double cell_area = (u_lo - u_hi) * (ph_hi - ph_lo);
  w[cell] = 1.0 - 0.5 * (area / cell_area);
}

// ---------------------------------------------------------------------------
// normalised associated Legendre functions
// ---------------------------------------------------------------------------
//
// Pbar_l^m = K_lm P_l^m with K_lm^2 = (2l+1)/(4 pi) (2 - delta_m0) (l-m)!/(l+m)!
// and the Condon-Shortley phase in P_l^m.  Standard normalised recurrences:
//   Pbar_0^0 = 1/sqrt(4 pi), Pbar_1^1 = -sqrt(3) s Pbar_0^0,
//   Pbar_m^m = -sqrt((2m+1)/(2m)) s Pbar_{m-1}^{m-1}  (m >= 2),
//   Pbar_{m+1}^m = sqrt(2m+3) x Pbar_m^m,
//   Pbar_l^m = a_lm (x Pbar_{l-1}^m - b_lm Pbar_{l-2}^m),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).

__device__ __forceinline__ double pbar_mm(int m, double s) {
  double p = 0.28209479177387814347403972578039;   // 1/sqrt(4 pi)
  if (m >= 1) p *= -sqrt(3.0) * s;
  for (int k = 2; k <= m; ++k) p *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
  return p;
}

// Walk l = m..lmax at fixed m, calling f(l, Pbar_l^m).
template <class F>
__device__ __forceinline__ void pbar_column(int m, int lmax, double x, double s, F f) {
  double p2 = 0.0;
  double p1 = pbar_mm(m, s);
  f(m, p1);
  if (m + 1 > lmax) return;
  double p0 = sqrt(2.0 * m + 3.0) * x * p1;
  f(m + 1, p0);
  for (int l = m + 2; l <= lmax; ++l) {
    p2 = p1;
    p1 = p0;
    const double ll = (double)l * l, mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
    const double a = sqrt((4.0 * ll - 1.0) / (ll - mm));
    const double b = sqrt((l1 - mm) / (4.0 * l1 - 1.0));
    p0 = a * (x * p1 - b * p2);
    f(l, p0);
  }
}

// ---------------------------------------------------------------------------
// K_lm T_j^(lm): one thread per (j, m); Gauss-Legendre in theta over the cell
// (the integrand sin(t) P_l^m(cos t) is a trigonometric polynomial of degree
// l + 1; lmax + 32 nodes integrate it to rounding).
// ---------------------------------------------------------------------------
__global__ void k_tbar(int n_theta, int lmax, int n_lm, double th0, double dth,
                       const double *__restrict__ gx, const double *__restrict__ gw, int nq,
                       double *__restrict__ tbar) {
  const int m = threadIdx.x;
  const int j = blockIdx.x;
  if (m > lmax || j >= n_theta) return;
  double acc[YY_LMAX_CAP + 1];
  for (int l = 0; l <= lmax; ++l) acc[l] = 0.0;
  const double a = th0 + dth * j;
  for (int q = 0; q < nq; ++q) {
    const double t = a + dth * gx[q];
    const double x = cos(t), s = sin(t);
    const double wq = dth * gw[q] * s;
    pbar_column(m, lmax, x, s, [&](int l, double p) { acc[l] += wq * p; });
  }
  for (int l = m; l <= lmax; ++l) {
    if (m == 0) {
      tbar[(size_t)j * n_lm + l * l] = acc[l];
    } else {
      tbar[(size_t)j * n_lm + l * l + 2 * m - 1] = acc[l];
      tbar[(size_t)j * n_lm + l * l + 2 * m] = acc[l];
    }
  }
}

__device__ __forceinline__ void mode_lm(int idx, int &l, int &m, bool &is_sin) {
  l = (int)sqrtf((float)idx);   // corrected below; exact for idx < 2^24
  while (l * l > idx) --l;
  while ((l + 1) * (l + 1) <= idx) ++l;
  const int r = idx - l * l;
  m = (r + 1) / 2;
  is_sin = (r > 0) && (r % 2 == 0);
}

// B_an[idx][jk] = w_jk K_lm T_j^(lm) {C_k^(m) | S_k^(m)}; C and S in the
// product forms 2 cos(m phi_c) sin(m dphi / 2) / m, 2 sin(m phi_c) sin(m dphi / 2) / m
// of the §2 closed forms.
__global__ void k_analysis_table(int n_theta, int n_phi, int n_lm, double ph0, double dph,
                                 const double *__restrict__ w, const double *__restrict__ tbar,
                                 double *__restrict__ ban) {
  const size_t n_ang = (size_t)n_theta * n_phi;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_ang * n_lm) return;
  const int idx = (int)(e / n_ang);
  const int jk = (int)(e % n_ang);
  const int j = jk / n_phi, k = jk % n_phi;
  int l, m;
  bool is_sin;
  mode_lm(idx, l, m, is_sin);
  double az;
  if (m == 0) {
    az = dph;
  } else {
    const double phc = ph0 + dph * (k + 0.5);
    const double half = 2.0 * sin(0.5 * m * dph) / m;
    az = is_sin ? sin(m * phc) * half : cos(m * phc) * half;
  }
  ban[e] = w[jk] * tbar[(size_t)j * n_lm + idx] * az;
}

// ---------------------------------------------------------------------------
// synthesis tables: one block per cell, one thread per m.
// ---------------------------------------------------------------------------
//
// Pole-safe derivatives of the normalised functions (Condon-Shortley phase):
//  dPbar_l^0/dtheta = sqrt(l(l+1)/2) Pbar_l^1
//  dPbar_l^m/dtheta = ( sqrt((l-m)(l+m+1)) Pbar_l^(m+1)
//                      - sqrt(d_m (l+m)(l-m+1)) Pbar_l^(m-1) ) / 2,  m >= 1
//  m Pbar_l^m / sin = -sqrt((2l+1)/(2l-1)) ( sqrt((l-m)(l-m-1)) Pbar_(l-1)^(m+1)
//                      + sqrt(d_m (l+m)(l+m-1)) Pbar_(l-1)^(m-1) ) / 2,  m >= 1
// with d_1 = 2, d_m = 1 otherwise (the 2 - delta_m0 factor of K).
// These follow from dP_l^m/dtheta = (P_l^(m+1) - (l+m)(l-m+1) P_l^(m-1)) / 2 and
// m P_l^m / sin = -(P_(l-1)^(m+1) + (l+m-1)(l+m) P_(l-1)^(m-1)) / 2.

__device__ __forceinline__ double tri_get(const double *P, int l, int m, int lmax) {
  if (l < 0 || m < 0 || m > l || l > lmax) return 0.0;
  return P[tri(l, m)];
}

__device__ __forceinline__ double dpbar(const double *P, int l, int m, int lmax) {
  if (l == 0) return 0.0;
  if (m == 0) return sqrt(0.5 * l * (l + 1.0)) * tri_get(P, l, 1, lmax);
  const double dm = (m == 1) ? 2.0 : 1.0;
  return 0.5 * (sqrt((double)(l - m) * (l + m + 1)) * tri_get(P, l, m + 1, lmax)
                - sqrt(dm * (l + m) * (l - m + 1.0)) * tri_get(P, l, m - 1, lmax));
}

__device__ __forceinline__ double mpbar_over_sin(const double *P, int l, int m, int lmax) {
  if (m == 0) return 0.0;
  const double dm = (m == 1) ? 2.0 : 1.0;
  const double f = sqrt((2.0 * l + 1.0) / (2.0 * l - 1.0));
  return -0.5 * f * (sqrt((double)(l - m) * (l - m - 1.0)) * tri_get(P, l - 1, m + 1, lmax)
                     + sqrt(dm * (l + m) * (l + m - 1.0)) * tri_get(P, l - 1, m - 1, lmax));
}

struct SynthGeom {
  double th0, ph0, dth, dph;
  int n_theta, n_phi, lmax, n_lm;
};

__global__ void k_synth_tables(SynthGeom G, double *__restrict__ ysyn, double *__restrict__ ysyn_t,
                               double *__restrict__ ysyn_p) {
  extern __shared__ double sm[];
  double *P = sm;
  const int cell = blockIdx.x;
  const int j = cell / G.n_phi, k = cell % G.n_phi;
  const double th = G.th0 + G.dth * (j + 0.5);
  const double ph = G.ph0 + G.dph * (k + 0.5);
  const double st = sin(th), ct = cos(th);
  for (int m = threadIdx.x; m <= G.lmax; m += blockDim.x)
    pbar_column(m, G.lmax, ct, st, [&](int l, double p) { P[tri(l, m)] = p; });
  __syncthreads();

  const size_t row = (size_t)cell * G.n_lm;
  for (int m = threadIdx.x; m <= G.lmax; m += blockDim.x) {
    const double cm = cos(m * ph), sm_ = sin(m * ph);
    for (int l = m; l <= G.lmax; ++l) {
      const double p = P[tri(l, m)];
      const double dp = dpbar(P, l, m, G.lmax);
      const double qs = mpbar_over_sin(P, l, m, G.lmax);
      if (m == 0) {
        const int idx = l * l;
        ysyn[row + idx] = p;
        ysyn_t[row + idx] = dp;
        ysyn_p[row + idx] = 0.0;
      } else {
        const int ic = l * l + 2 * m - 1, is = l * l + 2 * m;
        ysyn[row + ic] = p * cm;
        ysyn[row + is] = p * sm_;
        // d/dtheta, and (1/sin) d/dphi of cos(m phi) -> -m sin, sin(m phi) -> m cos
        ysyn_t[row + ic] = dp * cm;
        ysyn_t[row + is] = dp * sm_;
        ysyn_p[row + ic] = -qs * sm_;
        ysyn_p[row + is] = qs * cm;
      }
    }
  }
}

// Separable synthesis tables at the cell-centre colatitudes: one block per j,
// one thread per m.  P[j][idx] = K_lm P_l^m(cos theta_j), dP the theta
// derivative, Q the m P / sin theta factor of the phi derivative (the same
// value in the cos and sin slot of a mode); tr[t][k] = 1, cos(m phi_k),
// sin(m phi_k) for t = 0, 2m - 1, 2m at the cell-centre longitudes.
__global__ void k_sep_ptables(int n_theta, int lmax, int n_lm, double th0, double dth, double *__restrict__ P,
                              double *__restrict__ dP, double *__restrict__ Qs) {
  extern __shared__ double smt[];
  const int j = blockIdx.x;
  const double th = th0 + dth * (j + 0.5);
  const double st = sin(th), ct = cos(th);
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x)
    pbar_column(m, lmax, ct, st, [&](int l, double p) { smt[tri(l, m)] = p; });
  __syncthreads();
  const size_t row = (size_t)j * n_lm;
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    for (int l = m; l <= lmax; ++l) {
      const double p = smt[tri(l, m)], dp = dpbar(smt, l, m, lmax), qs = mpbar_over_sin(smt, l, m, lmax);
      const int i0 = (m == 0) ? l * l : l * l + 2 * m - 1;
      P[row + i0] = p;
      dP[row + i0] = dp;
      Qs[row + i0] = qs;
      if (m > 0) {
        P[row + i0 + 1] = p;
        dP[row + i0 + 1] = dp;
        Qs[row + i0 + 1] = qs;
      }
    }
  }
}

__global__ void k_sep_trig(int n_phi, int lmax, double ph0, double dph, double *__restrict__ tr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (2 * lmax + 1) * n_phi) return;
  const int t = e / n_phi, k = e % n_phi;
  const double ph = ph0 + dph * (k + 0.5);
  const int m = (t + 1) / 2;
  tr[e] = (t == 0) ? 1.0 : ((t & 1) ? cos(m * ph) : sin(m * ph));
}

// ---------------------------------------------------------------------------
// rotation of the other patch's harmonics
// ---------------------------------------------------------------------------
//
// A point with own-frame Cartesian direction v has direction M v in the other
// patch's frame, M (x, y, z) = (-x, z, y) (Eqs. trafotheta / trafophi); M is a
// rotation (by pi about (0, 1, 1) / sqrt 2) and its own inverse, so the same
// matrices serve both patches.  The real harmonics Y_i = K_lm P_l^m {cos, sin}
// are orthonormal on the sphere and a rotation keeps the degree, hence
//   Y_i(M v) = sum_j D^l_ij Y_j(v),   D^l_ij = int Y_i(M v) Y_j(v) dOmega,
// i, j over the 2l+1 modes of degree l in index order.  The integrand is a
// polynomial of degree 2l on the sphere: Gauss-Legendre in cos(theta) with
// lmax + 1 nodes times 2 lmax + 2 equispaced azimuths integrates it to
// rounding.  The harmonics of a batch of quadrature points are tabulated
// first (k_rot_points), then every D^l row accumulates over the batch
// (k_rot_accum).  Storage: D^l row-major at offset l (4l^2 - 1) / 3.

// One block per point of the batch: own-frame harmonics, and the other
// frame's harmonics times the quadrature weight.
__global__ void k_rot_points(int lmax, int n_lm, int n_az, int pt0, const double *__restrict__ gx,
                             const double *__restrict__ gw, double *__restrict__ y_own,
                             double *__restrict__ y_oth) {
  extern __shared__ double smp[];
  const int ntri = (lmax + 1) * (lmax + 2) / 2;
  double *Po = smp, *Px = smp + ntri;
  const int pt = pt0 + blockIdx.x;
  const int a = pt / n_az, c = pt % n_az;
  const double mu = 2.0 * gx[a] - 1.0;                   // nodes on [0, 1] mapped to [-1, 1]
  const double wq = 2.0 * gw[a] * (2.0 * kPi / n_az);
  const double ph = 2.0 * kPi * (c + 0.5) / n_az;
  const double s = sqrt(fmax(0.0, 1.0 - mu * mu));
  const double vx = s * cos(ph), vy = s * sin(ph), vz = mu;
  const double ox = -vx, oy = vz, oz = vy;
  const double so = sqrt(ox * ox + oy * oy);
  const double pho = atan2(oy, ox);
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    pbar_column(m, lmax, mu, s, [&](int l, double p) { Po[tri(l, m)] = p; });
    pbar_column(m, lmax, oz, so, [&](int l, double p) { Px[tri(l, m)] = p; });
  }
  __syncthreads();
  double *yo = y_own + (size_t)blockIdx.x * n_lm, *yx = y_oth + (size_t)blockIdx.x * n_lm;
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    const double cm = cos(m * ph), sm_ = sin(m * ph), cmo = cos(m * pho), smo = sin(m * pho);
    for (int l = m; l <= lmax; ++l) {
      const double po = Po[tri(l, m)], px = wq * Px[tri(l, m)];
      if (m == 0) {
        yo[l * l] = po;
        yx[l * l] = px;
      } else {
        yo[l * l + 2 * m - 1] = po * cm;
        yo[l * l + 2 * m] = po * sm_;
        yx[l * l + 2 * m - 1] = px * cmo;
        yx[l * l + 2 * m] = px * smo;
      }
    }
  }
}

// One block per mode row (l, i): D^l_ij (+)= sum over the batch of
// y_oth[pt][l^2 + i] y_own[pt][l^2 + j], points in ascending order.
__global__ void k_rot_accum(int n_lm, int n_pts, int first, const double *__restrict__ y_own,
                            const double *__restrict__ y_oth, double *__restrict__ rot) {
  const int row = blockIdx.x;
  int l, m;
  bool is_sin;
  mode_lm(row, l, m, is_sin);
  const int w = 2 * l + 1, i = row - l * l;
  double *D = rot + (size_t)l * (4 * l * l - 1) / 3 + (size_t)i * w;
  for (int j = threadIdx.x; j < w; j += blockDim.x) {
    double acc = first ? 0.0 : D[j];
    for (int p = 0; p < n_pts; ++p) acc = fma(y_oth[(size_t)p * n_lm + row], y_own[(size_t)p * n_lm + l * l + j], acc);
    D[j] = acc;
  }
}

// ---------------------------------------------------------------------------
// radial scan coefficients, one thread per (zone n, l)
// ---------------------------------------------------------------------------
//
// With zone n = [r_n, r_{n+1}] (r_n = r_edges[n]) and output radius r_{n+1}:
//   inner  c_n = a_n c_{n-1} + b_n A_n,   c_{-1} = 0
//          a_n = (r_n / r_{n+1})^(l+1),   b_n = r_{n+1}^-(l+1) R_in,n
//              = r_{n+1}^2 (1 - (r_n/r_{n+1})^(l+3)) / (l+3)
//   outer  d_n = e_n d_{n+1} + f_n A_{n+1},  d_{n_r - 1} = 0
//          e_n = (r_{n+1} / r_{n+2})^l,  f_n = r_{n+1}^l R_out,n+1
//              = r_{n+1}^2 ((r_{n+2}/r_{n+1})^(2-l) - 1) / (2 - l)   (l != 2)
//              = r_{n+1}^2 ln(r_{n+2}/r_{n+1})                       (l = 2)
// so c_n = r_{n+1}^-(l+1) sum_{i<=n} R_in,i A_i and d_n = r_{n+1}^l sum_{i>n}
// R_out,i A_i (Eqs. phiin / phiout), computed with expm1/log so that no
// power of r is formed explicitly.  Entries 4..7 turn (c_n, d_n) into the
// synthesis coefficients:  Q = k4 (c + d),  Q_r = k5 c + k6 d,  Q_t = k7 (c + d)
// (factors listed in the body).
__global__ void k_scan_coeffs(int n_r, int lmax, double G, const double *__restrict__ r,
                              double *__restrict__ coef) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_r * (lmax + 1)) return;
  const int n = e / (lmax + 1), l = e % (lmax + 1);
  const double r0 = r[n], r1 = r[n + 1];
  const double lq = (r0 > 0.0) ? log(r0 / r1) : -INFINITY;   // ln(r_n / r_{n+1}) <= 0
  const double a = exp((l + 1.0) * lq);
  const double b = r1 * r1 * (-expm1((l + 3.0) * lq)) / (l + 3.0);
  double ee = 0.0, f = 0.0;
  if (n + 1 < n_r) {
    const double r2 = r[n + 2];
    const double lu = log(r2 / r1);                          // > 0
    ee = exp(-(double)l * lu);
    f = (l == 2) ? r1 * r1 * lu : r1 * r1 * expm1((2.0 - l) * lu) / (2.0 - l);
  }
  const double fq = -G * 12.566370614359172953850573533118 / (2.0 * l + 1.0);
  const double inv_r = 1.0 / r1;
  double *o = coef + (size_t)e * 8;
  o[0] = a;
  o[1] = b;
  o[2] = ee;
  o[3] = f;
  o[4] = fq;                        // Phi:      -G 4pi/(2l+1) (c + d)
  o[5] = fq * (l + 1.0) * inv_r;    // g_r:       G 4pi/(2l+1) (-(l+1) c + l d) / r
  o[6] = -fq * l * inv_r;
  o[7] = -fq * inv_r;               // g_angle:   G 4pi/(2l+1) (c + d) / r
}

// w = 1: on the full spherical polar grid every cell is counted once
__global__ void k_unit_weights(int n, double *__restrict__ w) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) w[e] = 1.0;
}

__global__ void k_round_f32(int n, const double *__restrict__ src, float *__restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = (float)src[e];
}

}  // namespace

cudaError_t build_tables(yy_grid *g, const double *gl_host, int n_gl) {
  cudaError_t err;
  // GL tables on [0, 1]: [0, 32) nodes / [32, 64) weights for the weights
  // kernel; then n_gl nodes and weights for T; then lmax + 1 nodes and
  // weights for the rotation table.
  const int n_tab = 2 * YY_GL_WEIGHT_NODES + 2 * n_gl + 2 * (g->lmax + 1);
  if ((err = dmalloc((void **)&g->gl_nodes, n_tab * sizeof(double))) != cudaSuccess) return err;
  if ((err = cudaMemcpy(g->gl_nodes, gl_host, n_tab * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;

  WeightGeom wg;
  wg.th0 = g->th0;
  wg.ph0 = g->ph0;
  wg.dth = g->dth;
  wg.dph = g->dph;
  wg.c1 = cos(kPi / 4 - g->delta_theta);
  wg.t2 = tan(kPi / 4 - g->delta_phi);
  wg.n_theta = g->n_theta;
  wg.n_phi = g->n_phi;
  if (g->n_patch == 2)
    k_weights<<<(g->n_ang + 127) / 128, 128>>>(wg, g->gl_nodes, g->w);
  else
    k_unit_weights<<<(g->n_ang + 255) / 256, 256>>>(g->n_ang, g->w);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;

  const double *gx = g->gl_nodes + 2 * YY_GL_WEIGHT_NODES;
  const double *gw = gx + n_gl;
  cudaMemset(g->tbar, 0, (size_t)g->n_theta * g->n_lm * sizeof(double));
  k_tbar<<<g->n_theta, 128>>>(g->n_theta, g->lmax, g->n_lm, g->th0, g->dth, gx, gw, n_gl, g->tbar);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;

  const size_t n_ban = (size_t)g->n_ang * g->n_lm;
  k_analysis_table<<<(unsigned)((n_ban + 255) / 256), 256>>>(g->n_theta, g->n_phi, g->n_lm, g->ph0,
                                                             g->dph, g->w, g->tbar, g->ban);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;

  SynthGeom sg;
  sg.th0 = g->th0;
  sg.ph0 = g->ph0;
  sg.dth = g->dth;
  sg.dph = g->dph;
  sg.n_theta = g->n_theta;
  sg.n_phi = g->n_phi;
  sg.lmax = g->lmax;
  sg.n_lm = g->n_lm;
  const size_t smem = (size_t)(g->lmax + 1) * (g->lmax + 2) / 2 * sizeof(double);
  if ((err = cudaFuncSetAttribute(k_synth_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
    return err;
  k_synth_tables<<<g->n_ang, 96, smem>>>(sg, g->ysyn, g->ysyn_t, g->ysyn_p);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;

  if (g->n_patch == 2) {
    // rotation table: n_mu = lmax + 1 Gauss-Legendre nodes (after the T nodes) x 2 lmax + 2 azimuths
    const int n_mu = g->lmax + 1, n_az = 2 * g->lmax + 2, n_pts = n_mu * n_az;
    const double *mx = gx + 2 * n_gl, *mw = mx + n_mu;
    const size_t per_pt = (size_t)g->n_lm * sizeof(double);
    int batch = (int)std::min<size_t>((size_t)n_pts, (64u << 20) / (2 * per_pt));
    batch = std::max(batch, 1);
    double *yo = nullptr, *yx = nullptr;
    if ((err = dmalloc((void **)&yo, batch * per_pt)) != cudaSuccess) return err;
    if ((err = dmalloc((void **)&yx, batch * per_pt)) != cudaSuccess) {
      cudaFree(yo);
      return err;
    }
    const size_t psm = 2 * (size_t)(g->lmax + 1) * (g->lmax + 2) / 2 * sizeof(double);
    err = cudaFuncSetAttribute(k_rot_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    for (int p0 = 0; p0 < n_pts && err == cudaSuccess; p0 += batch) {
      const int nb = std::min(batch, n_pts - p0);
      k_rot_points<<<nb, 32, psm>>>(g->lmax, g->n_lm, n_az, p0, mx, mw, yo, yx);
      k_rot_accum<<<g->n_lm, 64>>>(g->n_lm, nb, p0 == 0 ? 1 : 0, yo, yx, g->rot);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    cudaFree(yo);
    cudaFree(yx);
    if (err != cudaSuccess) return err;
  }
  {
    const size_t psm = (size_t)(g->lmax + 1) * (g->lmax + 2) / 2 * sizeof(double);
    k_sep_ptables<<<g->n_theta, 32, psm>>>(g->n_theta, g->lmax, g->n_lm, g->th0, g->dth, g->sep_P, g->sep_dP,
                                           g->sep_Qs);
    const int n_tr = (2 * g->lmax + 1) * g->n_phi;
    k_sep_trig<<<(n_tr + 255) / 256, 256>>>(g->n_phi, g->lmax, g->ph0, g->dph, g->sep_tr);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if (g->n_patch == 2) {
    const int n_rot = rotation_table_size(g->lmax);
    k_round_f32<<<(n_rot + 255) / 256, 256>>>(n_rot, g->rot, g->rot32);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }

  const int n_sc = g->n_r * (g->lmax + 1);
  k_scan_coeffs<<<(n_sc + 127) / 128, 128>>>(g->n_r, g->lmax, g->G, g->r_edges, g->scan);
  return cudaGetLastError();
}

}  // namespace yy
