// Oracle: a plain, slow, FP64 CPU solver of the coupled Cahn-Hilliard /
// Allen-Cahn phase-field model of Boccardo et al., "Efficiency and accuracy of
// GPU-parallelized Fourier spectral methods for solving phase-field models"
// (arXiv 2306.04322).
//
// TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
// CUDA path is compared against.  It shares no code, header, table or helper
// with the CUDA library; only the test suite, the smoke check and the CPU
// baseline leg of the benchmark may load it.  The product path never calls it.
//
// Everything here follows the paper's equations directly:
//   * free energy, Eq. (fe) and the definitions of f_chem, h and g in
//     Section 2.1 ("Problem formulation");
//   * semi-implicit time discretisation, Eqs. (C-H_discrete), (A-C_discrete);
//   * Fourier-space solve, Eqs. (C-H_discrete_fft), (A-C_discrete_fft), the
//     independent terms (C-H_fft_b), (A-C_fft_b) and the per-mode inversion
//     (A-C_discrete_fft_c), (A-C_discrete_fft_eta);
//   * frequency vectors, Eqs. (Gamma_fft), (Gamma_fft_3d) and the FS-FD
//     redefinitions (Gamma_fft-fdO2), (Gamma_fft-fdO4) and their 3D forms;
//   * Algorithm 1 (FS solution algorithm), taken step by step;
//   * the explicit finite-difference comparison scheme of Section 2.2
//     (forward Euler, 5-point / 7-point Laplacian, periodic boundaries).
// The adjoint of one step is not in the paper; it is the transpose of the
// Jacobian of the Algorithm-1 step map, written out plainly below.
//
// Precision: FP64 throughout, FFT twiddles from long-double cos/sin of the
// exactly reduced angle 2*pi*k/n (one table per transform length, no
// recurrences).  Compiled with -ffp-contract=off so no FMA contraction
// changes the rounding of the written expressions.
//
// Data layout: a field is a contiguous array of N = nx*ny*nz doubles with x
// fastest, idx = (z*ny + y)*nx + x.  A state is nf = 1 + p such arrays in the
// order c, eta_1 .. eta_p.

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Model and grid parameters (Section 2.1 and Algorithm 1 initialisation).
typedef struct {
  int ndim;          // 2 or 3
  int n[3];          // grid points along x, y, z (n[2] = 1 in 2D)
  double dx[3];      // grid spacing along x, y, z
  int p;             // number of order parameters eta_i
  double M, L, kappa_c, kappa_eta, rho2, c_alpha, c_beta, w, alpha, dt;
  int lap;           // 0: spectral |xi|^2, 1: FS-FD O(dl^2), 2: FS-FD O(dl^4)
} or_params;

}  // extern "C"

namespace {

const long double kPiL = 3.141592653589793238462643383279502884L;

struct Cplx {
  double re, im;
};

inline Cplx cmul(Cplx a, Cplx b) {
  return Cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
inline Cplx cadd(Cplx a, Cplx b) { return Cplx{a.re + b.re, a.im + b.im}; }
inline Cplx csub(Cplx a, Cplx b) { return Cplx{a.re - b.re, a.im - b.im}; }

// Twiddles exp(sign * 2*pi*i*k/n) for k = 0..n/2-1, each from its own exactly
// reduced angle in long double.
std::vector<Cplx> twiddles(int n, int sign) {
  std::vector<Cplx> t(n / 2 > 0 ? n / 2 : 1);
  for (int k = 0; k < n / 2; ++k) {
    long double ang = 2.0L * kPiL * (long double)k / (long double)n;
    t[k].re = (double)cosl(ang);
    t[k].im = (double)(sign * sinl(ang));
  }
  return t;
}

// In-place iterative radix-2 Cooley-Tukey DFT of length n (a power of two):
// X[k] = sum_j x[j] exp(sign * 2*pi*i*j*k/n), unnormalised.
void fft1d(Cplx* a, int n, const std::vector<Cplx>& tw) {
  for (int i = 1, j = 0; i < n; ++i) {  // bit-reversal permutation
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      Cplx t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len / 2, step = n / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < half; ++k) {
        Cplx u = a[i + k];
        Cplx v = cmul(a[i + k + half], tw[k * step]);
        a[i + k] = cadd(u, v);
        a[i + k + half] = csub(u, v);
      }
  }
}

// Multi-dimensional unnormalised DFT along every axis of a complex grid.
void fftnd(Cplx* a, const int* n, int ndim, int sign) {
  long N = 1;
  for (int d = 0; d < ndim; ++d) N *= n[d];
  long stride = 1;
  for (int d = 0; d < ndim; ++d) {
    int len = n[d];
    if (len > 1) {
      std::vector<Cplx> tw = twiddles(len, sign);
      long nlines = N / len;
#pragma omp parallel
      {
        std::vector<Cplx> line(len);
#pragma omp for schedule(static)
        for (long l = 0; l < nlines; ++l) {
          long outer = l / stride, inner = l % stride;
          long base = outer * stride * len + inner;
          for (int j = 0; j < len; ++j) line[j] = a[base + (long)j * stride];
          fft1d(line.data(), len, tw);
          for (int j = 0; j < len; ++j) a[base + (long)j * stride] = line[j];
        }
      }
    }
    stride *= len;
  }
}

long npoints(const or_params* P) {
  long N = 1;
  for (int d = 0; d < P->ndim; ++d) N *= P->n[d];
  return N;
}

// Integer frequency index of DFT bin k for length n, following the vector
// [0, ..., n/2, -(n/2-1), ..., -1] of Eq. (Gamma_fft).
int freq_index(int k, int n) { return k <= n / 2 ? k : k - n; }

// Per-axis contribution to the squared frequency norm.
//  lap 0: (2*pi*n_d/l_d)^2, Eqs. (Gamma_fft), (Gamma_fft_3d), l_d = n*dx.
//  lap 1: -2 (cos(dx xi) - 1)/dx^2, Eqs. (Gamma_fft-fdO2), (..._3d).
//  lap 2: -(16 cos(dx xi) - cos(2 dx xi) - 15)/(6 dx^2), Eqs. (Gamma_fft-fdO4).
double axis_k2(const or_params* P, int d, int k) {
  int n = P->n[d];
  double dx = P->dx[d];
  double l = n * dx;
  double xi = 2.0 * (double)kPiL * (double)freq_index(k, n) / l;
  if (P->lap == 1) return -2.0 * (std::cos(dx * xi) - 1.0) / (dx * dx);
  if (P->lap == 2)
    return -(16.0 * std::cos(dx * xi) - std::cos(2.0 * dx * xi) - 15.0) / (6.0 * dx * dx);
  return xi * xi;
}

// |xi|^2 on the full grid (Algorithm 1, built once before the time loop).
std::vector<double> build_k2(const or_params* P) {
  long N = npoints(P);
  std::vector<double> K2(N);
  int nx = P->n[0], ny = P->ndim > 1 ? P->n[1] : 1, nz = P->ndim > 2 ? P->n[2] : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double s = axis_k2(P, 0, x);
        if (P->ndim > 1) s += axis_k2(P, 1, y);
        if (P->ndim > 2) s += axis_k2(P, 2, z);
        K2[((long)z * ny + y) * nx + x] = s;
      }
  return K2;
}

// h(eta) = eta^3 (6 eta^2 - 15 eta + 10) and its first two derivatives.
double h_of(double e) { return e * e * e * (6.0 * e * e - 15.0 * e + 10.0); }
double dh_of(double e) { return 30.0 * e * e * e * e - 60.0 * e * e * e + 30.0 * e * e; }
double d2h_of(double e) { return 120.0 * e * e * e - 180.0 * e * e + 60.0 * e; }

}  // namespace

extern "C" {

// Chemical free-energy density f_chem = f_a (1 - h) + f_b h + w g at one point
// (Section 2.1): f_a = rho2 (c - c_alpha)^2, f_b = rho2 (c_beta - c)^2,
// h = sum_i h(eta_i), g = sum_i eta_i^2 (1 - eta_i)^2
//                        + alpha sum_i sum_{j != i} eta_i^2 eta_j^2.
double or_fchem_point(const or_params* P, double c, const double* eta) {
  double fa = P->rho2 * (c - P->c_alpha) * (c - P->c_alpha);
  double fb = P->rho2 * (P->c_beta - c) * (P->c_beta - c);
  double h = 0.0, g = 0.0;
  for (int i = 0; i < P->p; ++i) {
    h += h_of(eta[i]);
    g += eta[i] * eta[i] * (1.0 - eta[i]) * (1.0 - eta[i]);
  }
  for (int i = 0; i < P->p; ++i)
    for (int j = 0; j < P->p; ++j)
      if (j != i) g += P->alpha * eta[i] * eta[i] * eta[j] * eta[j];
  return fa * (1.0 - h) + fb * h + P->w * g;
}

// First derivatives of f_chem at one point: out[0] = df/dc, out[1+i] = df/deta_i.
// The double sum in g runs over ordered pairs (i, j), j != i, so each
// unordered pair appears twice; its derivative is accumulated term by term.
void or_dfchem_point(const or_params* P, double c, const double* eta, double* out) {
  double h = 0.0;
  for (int i = 0; i < P->p; ++i) h += h_of(eta[i]);
  double dfa = 2.0 * P->rho2 * (c - P->c_alpha);
  double dfb = -2.0 * P->rho2 * (P->c_beta - c);
  out[0] = dfa * (1.0 - h) + dfb * h;
  double fa = P->rho2 * (c - P->c_alpha) * (c - P->c_alpha);
  double fb = P->rho2 * (P->c_beta - c) * (P->c_beta - c);
  for (int k = 0; k < P->p; ++k) {
    double e = eta[k];
    double dg = 2.0 * e * (1.0 - e) * (1.0 - e) - 2.0 * e * e * (1.0 - e);
    for (int i = 0; i < P->p; ++i)
      for (int j = 0; j < P->p; ++j) {
        if (j == i) continue;
        if (i == k) dg += P->alpha * 2.0 * eta[i] * eta[j] * eta[j];
        if (j == k) dg += P->alpha * eta[i] * eta[i] * 2.0 * eta[j];
      }
    out[1 + k] = (fb - fa) * dh_of(e) + P->w * dg;
  }
}

// Second derivatives of f_chem at one point, row-major nf x nf, variables
// ordered (c, eta_1 .. eta_p).  Used only by the adjoint.
void or_d2fchem_point(const or_params* P, double c, const double* eta, double* H) {
  int nf = 1 + P->p;
  for (int a = 0; a < nf * nf; ++a) H[a] = 0.0;
  // d2/dc2 of f_a (1-h) + f_b h = 2 rho2 (1 - h) + 2 rho2 h
  {
    double h = 0.0;
    for (int i = 0; i < P->p; ++i) h += h_of(eta[i]);
    H[0] = 2.0 * P->rho2 * (1.0 - h) + 2.0 * P->rho2 * h;
  }
  double dfa = 2.0 * P->rho2 * (c - P->c_alpha);
  double dfb = -2.0 * P->rho2 * (P->c_beta - c);
  double fa = P->rho2 * (c - P->c_alpha) * (c - P->c_alpha);
  double fb = P->rho2 * (P->c_beta - c) * (P->c_beta - c);
  for (int k = 0; k < P->p; ++k) {
    double e = eta[k];
    double hck = (dfb - dfa) * dh_of(e);  // d2 f / dc deta_k
    H[0 * nf + 1 + k] = hck;
    H[(1 + k) * nf + 0] = hck;
    for (int l = 0; l < P->p; ++l) {
      double v = 0.0;
      if (l == k) {
        v += (fb - fa) * d2h_of(e);
        v += P->w * (2.0 * (1.0 - e) * (1.0 - e) - 8.0 * e * (1.0 - e) + 2.0 * e * e);
      }
      // alpha sum over ordered pairs (i, j), j != i, of eta_i^2 eta_j^2
      for (int i = 0; i < P->p; ++i)
        for (int j = 0; j < P->p; ++j) {
          if (j == i) continue;
          // d2/deta_k deta_l of eta_i^2 eta_j^2
          double t = 0.0;
          if (i == k && i == l) t += 2.0 * eta[j] * eta[j];
          if (j == k && j == l) t += 2.0 * eta[i] * eta[i];
          if (i == k && j == l) t += 4.0 * eta[i] * eta[j];
          if (j == k && i == l) t += 4.0 * eta[i] * eta[j];
          v += P->w * P->alpha * t;
        }
      H[(1 + k) * nf + 1 + l] = v;
    }
  }
}

// Unnormalised multi-dimensional DFT of an interleaved complex array
// (re, im pairs), sign -1 forward, +1 backward.  Exposed for the FFT pins.
void or_fft(double* data, int ndim, const int* n, int sign) {
  fftnd(reinterpret_cast<Cplx*>(data), n, ndim, sign);
}

// |xi|^2 on the full grid, for the tests.
void or_k2(const or_params* P, double* out) {
  std::vector<double> K2 = build_k2(P);
  std::memcpy(out, K2.data(), K2.size() * sizeof(double));
}

// Pointwise derivative fields: out holds nf arrays (df/dc, df/deta_1..p).
void or_derivatives(const or_params* P, const double* fields, double* out) {
  long N = npoints(P);
  int nf = 1 + P->p;
  std::vector<double> eta(P->p > 0 ? P->p : 1), d(nf);
  for (long i = 0; i < N; ++i) {
    for (int k = 0; k < P->p; ++k) eta[k] = fields[(1 + k) * N + i];
    or_dfchem_point(P, fields[i], eta.data(), d.data());
    for (int f = 0; f < nf; ++f) out[f * N + i] = d[f];
  }
}

// Algorithm 1, nsteps iterations, in place on the real state `fields`
// (nf arrays).  The state carried between steps is the real fields; the
// Fourier transforms of c and eta_i at time t are recomputed from them at the
// top of each step.  Returns the largest |imaginary part| / max|real part|
// seen after an inverse transform (it must be at rounding level).
double or_step(const or_params* P, double* fields, int nsteps) {
  long N = npoints(P);
  int nf = 1 + P->p;
  int nfull[3] = {P->n[0], P->ndim > 1 ? P->n[1] : 1, P->ndim > 2 ? P->n[2] : 1};
  std::vector<double> K2 = build_k2(P);
  std::vector<double> deriv((size_t)nf * N);
  std::vector<Cplx> uhat(N), fhat(N);
  double worst_imag = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    // df_chem/dc and df_chem/deta_i at time t (explicit part).
    or_derivatives(P, fields, deriv.data());
    for (int f = 0; f < nf; ++f) {
      double* u = fields + (long)f * N;
      const double* fd = deriv.data() + (long)f * N;
      for (long i = 0; i < N; ++i) {
        uhat[i] = Cplx{u[i], 0.0};
        fhat[i] = Cplx{fd[i], 0.0};
      }
      fftnd(uhat.data(), nfull, P->ndim, -1);  // F of the field at time t
      fftnd(fhat.data(), nfull, P->ndim, -1);  // F of its derivative
      double X = (f == 0) ? P->M : P->L;
      double kap = (f == 0) ? P->kappa_c : P->kappa_eta;
      for (long i = 0; i < N; ++i) {
        double k2 = K2[i];
        Cplx b;
        double lhs;
        if (f == 0) {
          // b_c = c^ - M dt |xi|^2 (df/dc)^ ; (1 + M dt kappa_c |xi|^4) c^ = b_c
          b = Cplx{uhat[i].re - X * P->dt * k2 * fhat[i].re,
                   uhat[i].im - X * P->dt * k2 * fhat[i].im};
          lhs = 1.0 + X * P->dt * kap * k2 * k2;
        } else {
          // b_eta = eta^ - L dt (df/deta)^ ; (1 + L dt kappa_eta |xi|^2) eta^ = b_eta
          b = Cplx{uhat[i].re - X * P->dt * fhat[i].re, uhat[i].im - X * P->dt * fhat[i].im};
          lhs = 1.0 + X * P->dt * kap * k2;
        }
        uhat[i] = Cplx{b.re / lhs, b.im / lhs};
      }
      fftnd(uhat.data(), nfull, P->ndim, +1);  // F^-1 (scaled by 1/N below)
      double maxre = 0.0, maxim = 0.0;
      for (long i = 0; i < N; ++i) {
        u[i] = uhat[i].re / (double)N;
        maxre = std::fmax(maxre, std::fabs(u[i]));
        maxim = std::fmax(maxim, std::fabs(uhat[i].im / (double)N));
      }
      if (maxre > 0.0) worst_imag = std::fmax(worst_imag, maxim / maxre);
    }
  }
  return worst_imag;
}

// Total free energy, Eq. (fe), integrated with the rectangle rule over the
// periodic grid (dV = prod dx).  The gradient terms sum_x |grad phi|^2 use the
// same frequency vector as the scheme, through Parseval's identity
// sum_x |grad phi|^2 = (1/N) sum_k |xi|^2 |phi^(k)|^2.
// parts (optional, 2 + p entries): chemical, c-gradient, eta_i-gradient terms.
double or_free_energy(const or_params* P, const double* fields, double* parts) {
  long N = npoints(P);
  int nfull[3] = {P->n[0], P->ndim > 1 ? P->n[1] : 1, P->ndim > 2 ? P->n[2] : 1};
  double dV = 1.0;
  for (int d = 0; d < P->ndim; ++d) dV *= P->dx[d];
  std::vector<double> eta(P->p > 0 ? P->p : 1);
  double chem = 0.0;
  for (long i = 0; i < N; ++i) {
    for (int k = 0; k < P->p; ++k) eta[k] = fields[(1 + k) * N + i];
    chem += or_fchem_point(P, fields[i], eta.data());
  }
  chem *= dV;
  std::vector<double> K2 = build_k2(P);
  std::vector<Cplx> a(N);
  double total = chem;
  if (parts) parts[0] = chem;
  for (int f = 0; f < 1 + P->p; ++f) {
    for (long i = 0; i < N; ++i) a[i] = Cplx{fields[(long)f * N + i], 0.0};
    fftnd(a.data(), nfull, P->ndim, -1);
    double s = 0.0;
    for (long i = 0; i < N; ++i) s += K2[i] * (a[i].re * a[i].re + a[i].im * a[i].im);
    double kap = (f == 0) ? P->kappa_c : P->kappa_eta;
    double term = 0.5 * kap * s / (double)N * dV;
    if (parts) parts[1 + f] = term;
    total += term;
  }
  return total;
}

// Explicit finite-difference comparison scheme (Section 2.2): forward Euler in
// time, 5-point (2D) / 7-point (3D) Laplacian, periodic boundaries, three
// stages per step: (i) mu = df/dc - kappa_c lap(c); (ii) c += dt M lap(mu);
// (iii) eta_i += -dt L (df/deta_i - kappa_eta lap(eta_i)).
void or_fd_step(const or_params* P, double* fields, int nsteps) {
  long N = npoints(P);
  int nf = 1 + P->p;
  int nx = P->n[0], ny = P->ndim > 1 ? P->n[1] : 1, nz = P->ndim > 2 ? P->n[2] : 1;
  std::vector<double> deriv((size_t)nf * N), mu(N), old((size_t)nf * N);
  auto lap = [&](const double* a, long i) {
    long x = i % nx, y = (i / nx) % ny, z = i / ((long)nx * ny);
    double s = 0.0;
    long xm = (x + nx - 1) % nx, xp = (x + 1) % nx;
    s += (a[(z * ny + y) * nx + xm] - 2.0 * a[i] + a[(z * ny + y) * nx + xp]) / (P->dx[0] * P->dx[0]);
    if (P->ndim > 1) {
      long ym = (y + ny - 1) % ny, yp = (y + 1) % ny;
      s += (a[(z * ny + ym) * nx + x] - 2.0 * a[i] + a[(z * ny + yp) * nx + x]) / (P->dx[1] * P->dx[1]);
    }
    if (P->ndim > 2) {
      long zm = (z + nz - 1) % nz, zp = (z + 1) % nz;
      s += (a[(zm * ny + y) * nx + x] - 2.0 * a[i] + a[(zp * ny + y) * nx + x]) / (P->dx[2] * P->dx[2]);
    }
    return s;
  };
  for (int s = 0; s < nsteps; ++s) {
    std::memcpy(old.data(), fields, sizeof(double) * nf * N);
    or_derivatives(P, old.data(), deriv.data());
    for (long i = 0; i < N; ++i) mu[i] = deriv[i] - P->kappa_c * lap(old.data(), i);
    for (long i = 0; i < N; ++i) fields[i] = old[i] + P->dt * P->M * lap(mu.data(), i);
    for (int k = 0; k < P->p; ++k) {
      const double* e = old.data() + (long)(1 + k) * N;
      for (long i = 0; i < N; ++i)
        fields[(long)(1 + k) * N + i] =
            e[i] - P->dt * P->L * (deriv[(long)(1 + k) * N + i] - P->kappa_eta * lap(e, i));
    }
  }
}

// Adjoint of one Algorithm-1 step.  The step maps the real state u to
//   u'_phi = F^-1[ D1_phi F u_phi + D2_phi F f_phi(u) ],
// with, from Eqs. (C-H_discrete_fft)..(A-C_discrete_fft_eta),
//   c:     D1 = 1/(1 + M dt kc K2^2),  D2 = -M dt K2 / (1 + M dt kc K2^2)
//   eta_i: D1 = 1/(1 + L dt ke K2),    D2 = -L dt / (1 + L dt ke K2)
// and f_phi = df_chem/dphi.  Both D are real and even in k, so F^-1 D F is a
// real symmetric operator; the Jacobian is J = G1 + G2 H(u) with H the
// pointwise Hessian of f_chem, and its transpose acts as
//   lam_phi = G1_phi lam'_phi + sum_psi H_phi,psi(u) (G2_psi lam'_psi).
// Parameter sensitivities: grad[t] += <lam', d u' / d theta_t> for
// theta = (M, L, kappa_c, kappa_eta), each dD/dtheta written out below.
void or_adjoint_step(const or_params* P, const double* u, const double* lam_in,
                     double* lam_out, double* grad) {
  long N = npoints(P);
  int nf = 1 + P->p;
  int nfull[3] = {P->n[0], P->ndim > 1 ? P->n[1] : 1, P->ndim > 2 ? P->n[2] : 1};
  std::vector<double> K2 = build_k2(P);
  std::vector<double> deriv((size_t)nf * N);
  or_derivatives(P, u, deriv.data());
  std::vector<double> G1l((size_t)nf * N), G2l((size_t)nf * N);
  std::vector<Cplx> L(N), a(N), b(N), U(N), Fh(N);
  double dt = P->dt;
  for (int f = 0; f < nf; ++f) {
    for (long i = 0; i < N; ++i) {
      L[i] = Cplx{lam_in[(long)f * N + i], 0.0};
      U[i] = Cplx{u[(long)f * N + i], 0.0};
      Fh[i] = Cplx{deriv[(long)f * N + i], 0.0};
    }
    fftnd(L.data(), nfull, P->ndim, -1);
    fftnd(U.data(), nfull, P->ndim, -1);
    fftnd(Fh.data(), nfull, P->ndim, -1);
    double g[4] = {0, 0, 0, 0};
    for (long i = 0; i < N; ++i) {
      double k2 = K2[i];
      double d1, d2, dd1[4] = {0, 0, 0, 0}, dd2[4] = {0, 0, 0, 0};
      if (f == 0) {
        double den = 1.0 + P->M * dt * P->kappa_c * k2 * k2;
        d1 = 1.0 / den;
        d2 = -P->M * dt * k2 / den;
        dd1[0] = -dt * P->kappa_c * k2 * k2 / (den * den);        // dD1/dM
        dd1[2] = -P->M * dt * k2 * k2 / (den * den);              // dD1/dkappa_c
        dd2[0] = -dt * k2 / den + P->M * dt * k2 * dt * P->kappa_c * k2 * k2 / (den * den);
        dd2[2] = P->M * dt * k2 * P->M * dt * k2 * k2 / (den * den);
      } else {
        double den = 1.0 + P->L * dt * P->kappa_eta * k2;
        d1 = 1.0 / den;
        d2 = -P->L * dt / den;
        dd1[1] = -dt * P->kappa_eta * k2 / (den * den);           // dD1/dL
        dd1[3] = -P->L * dt * k2 / (den * den);                   // dD1/dkappa_eta
        dd2[1] = -dt / den + P->L * dt * dt * P->kappa_eta * k2 / (den * den);
        dd2[3] = P->L * dt * P->L * dt * k2 / (den * den);
      }
      a[i] = Cplx{d1 * L[i].re, d1 * L[i].im};
      b[i] = Cplx{d2 * L[i].re, d2 * L[i].im};
      // Parseval: sum_x lam'(x) (F^-1 X)(x) = (1/N) sum_k conj(L(k)) X(k)
      for (int t = 0; t < 4; ++t) {
        double xr = dd1[t] * U[i].re + dd2[t] * Fh[i].re;
        double xi = dd1[t] * U[i].im + dd2[t] * Fh[i].im;
        g[t] += L[i].re * xr + L[i].im * xi;
      }
    }
    if (grad)
      for (int t = 0; t < 4; ++t) grad[t] += g[t] / (double)N;
    fftnd(a.data(), nfull, P->ndim, +1);
    fftnd(b.data(), nfull, P->ndim, +1);
    for (long i = 0; i < N; ++i) {
      G1l[(long)f * N + i] = a[i].re / (double)N;
      G2l[(long)f * N + i] = b[i].re / (double)N;
    }
  }
  std::vector<double> eta(P->p > 0 ? P->p : 1), H((size_t)nf * nf);
  for (long i = 0; i < N; ++i) {
    for (int k = 0; k < P->p; ++k) eta[k] = u[(long)(1 + k) * N + i];
    or_d2fchem_point(P, u[i], eta.data(), H.data());
    for (int ph = 0; ph < nf; ++ph) {
      double s = G1l[(long)ph * N + i];
      for (int ps = 0; ps < nf; ++ps) s += H[ph * nf + ps] * G2l[(long)ps * N + i];
      lam_out[(long)ph * N + i] = s;
    }
  }
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

}  // extern "C"
