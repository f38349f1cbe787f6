/*
 * ffe_oracle.c -- plain FP64 CPU oracle for the grand free energy of the
 * two-band iron-pnictide model with intra-band Fulde-Ferrell pairing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Everything here is the literal definition, evaluated in IEEE double with
 * libm, without blocking, fusion or algebraic rearrangement beyond what the
 * paper writes down:
 *
 *   Band energies (App. A, two-band model of Raghu et al.):
 *     T11(k) = -2 (t1 cos kx + t2 cos ky) - 4 t3 cos kx cos ky
 *     T22(k) = -2 (t2 cos kx + t1 cos ky) - 4 t3 cos kx cos ky
 *     T12(k) = -4 t4 sin kx sin ky
 *     E_{+/-}(k) = (T11+T22)/2 +/- sqrt(((T11-T22)/2)^2 + T12^2)
 *   Spin-resolved energies (Sec. 2, T_{k sigma} = T_k - (mu + sigma h)),
 *   sigma(up) = +1:
 *     E_{eps,k,up}        = E_eps(k + Q/2)  - mu - h
 *     E_{eps,-k+Q/2,down} = E_eps(-k + Q/2) - mu + h
 *   Quasiparticle energies (Sec. 2, Eq. enequasiparticle):
 *     Ep/m = (E_up - E_dn)/2 +/- sqrt(((E_up + E_dn)/2)^2 + |Delta eta(k)|^2)
 *   Free energy per band (Sec. 2, Eq. freeene), read with a + sign and
 *   coefficient 1/U on the pairing term (the printed "- 2|Delta|^2/V" makes
 *   Omega decrease monotonically in Delta; the + sign reproduces the BCS gap
 *   equation, which the tests check):
 *     Omega_eps = sum_k [ F(Ep) + F(Em) + E_dn + Delta^2 / U ],
 *     F(E) = -T ln(1 + exp(-E/T)).
 *   Omega = Omega_- + Omega_+.
 *   k runs over the unshifted N x N lattice k = 2 pi (i, j) / N.
 *   Form factor eta(k) = eta_amp cos kx cos ky (s+- symmetry, Sec. 1).
 *
 * The k-sum is Neumaier-compensated.  Batches parallelise over points with
 * OpenMP (the paper's CPU code parallelises over the Delta loop, Sec. 3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double t1, t2, t3, t4, mu; /* hopping parameters and chemical potential */
  double eta_amp;            /* amplitude of the s+- form factor          */
  double U;                  /* pairing strength: term +Delta^2/U per k    */
  double U_band[2];          /* per-band coupling V_eps of Sec. 2 (read as
                                U_eps): > 0 replaces U in band eps's term  */
} ffeo_model;

/* The coupling of band b: its own U_eps where one is given, else U. */
static double band_U(const ffeo_model* m, int b) {
  return m->U_band[b] > 0.0 ? m->U_band[b] : m->U;
}

/* Neumaier (improved Kahan-Babuska) running sum. */
typedef struct {
  double s, c;
} nsum;

static void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

static double nsum_value(const nsum* a) { return a->s + a->c; }

/* App. A: the two eigenvalues of the 2x2 hopping matrix at momentum (kx, ky).
 * e[0] = E_-(k) (hole-like), e[1] = E_+(k) (electron-like). */
void ffeo_band_energies(const ffeo_model* m, double kx, double ky, double* e) {
  double cx = cos(kx), cy = cos(ky), sx = sin(kx), sy = sin(ky);
  double t11 = -2.0 * (m->t1 * cx + m->t2 * cy) - 4.0 * m->t3 * cx * cy;
  double t22 = -2.0 * (m->t2 * cx + m->t1 * cy) - 4.0 * m->t3 * cx * cy;
  double t12 = -4.0 * m->t4 * sx * sy;
  double mean = 0.5 * (t11 + t22);
  double half = 0.5 * (t11 - t22);
  double root = sqrt(half * half + t12 * t12);
  e[0] = mean - root;
  e[1] = mean + root;
}

/* Eq. enequasiparticle: the two Bogoliubov quasiparticle energies of one
 * (k up, -k+q down) pair with pairing amplitude gap = Delta * eta(k). */
void ffeo_quasiparticle(double e_up, double e_dn, double gap, double* ep,
                        double* em) {
  double d = 0.5 * (e_up - e_dn);
  double s = 0.5 * (e_up + e_dn);
  double r = sqrt(s * s + gap * gap);
  *ep = d + r;
  *em = d - r;
}

/* F(E) = -T ln(1 + exp(-E/T)), evaluated without overflow:
 * for E < 0, ln(1 + e^{-E/T}) = -E/T + ln(1 + e^{E/T}). */
double ffeo_F(double E, double T) {
  if (E >= 0.0) return -T * log1p(exp(-E / T));
  return E - T * log1p(exp(E / T));
}

/* Eq. freeene summed over the k lattice for both bands.
 * omega_band (may be NULL) receives Omega_- and Omega_+. */
void ffeo_omega(const ffeo_model* m, int N, double qx, double qy, double h,
                double T, double delta, double* omega, double* omega_band) {
  nsum tot = {0.0, 0.0};
  nsum band[2] = {{0.0, 0.0}, {0.0, 0.0}};
  const double two_pi = 2.0 * M_PI;
  for (int j = 0; j < N; ++j) {
    double ky = two_pi * (double)j / (double)N;
    for (int i = 0; i < N; ++i) {
      double kx = two_pi * (double)i / (double)N;
      double e_kq[2], e_mkq[2];
      /* E_eps(k + Q/2) for spin up, E_eps(-k + Q/2) for spin down */
      ffeo_band_energies(m, kx + 0.5 * qx, ky + 0.5 * qy, e_kq);
      ffeo_band_energies(m, -kx + 0.5 * qx, -ky + 0.5 * qy, e_mkq);
      double eta = m->eta_amp * cos(kx) * cos(ky);
      for (int b = 0; b < 2; ++b) {
        double e_up = e_kq[b] - m->mu - h;
        double e_dn = e_mkq[b] - m->mu + h;
        double ep, em;
        ffeo_quasiparticle(e_up, e_dn, delta * eta, &ep, &em);
        double term = ffeo_F(ep, T) + ffeo_F(em, T) + e_dn + delta * delta / band_U(m, b);
        nsum_add(&tot, term);
        nsum_add(&band[b], term);
      }
    }
  }
  *omega = nsum_value(&tot);
  if (omega_band) {
    omega_band[0] = nsum_value(&band[0]);
    omega_band[1] = nsum_value(&band[1]);
  }
}

/* Eq. freeene for a model of nb bands whose band energies are given:
 * e_up[(j*N + i)*nb + b] = E_b(k + Q/2), e_dn[...] = E_b(-k + Q/2) for
 * k = 2 pi (i, j)/N (the three-band model of App. B, whose 3x3 hopping matrix
 * the caller diagonalises); U[b] is band b's coupling.  omega_band (may be
 * NULL) receives Omega_b. */
void ffeo_omega_given(int nb, int N, const double* e_up, const double* e_dn,
                      double eta_amp, double mu, const double* U, double h, double T,
                      double delta, double* omega, double* omega_band) {
  nsum tot = {0.0, 0.0};
  nsum band[8];
  for (int b = 0; b < nb; ++b) band[b].s = band[b].c = 0.0;
  const double two_pi = 2.0 * M_PI;
  for (int j = 0; j < N; ++j) {
    double ky = two_pi * (double)j / (double)N;
    for (int i = 0; i < N; ++i) {
      double kx = two_pi * (double)i / (double)N;
      double eta = eta_amp * cos(kx) * cos(ky);
      const int64_t base = ((int64_t)j * N + i) * nb;
      for (int b = 0; b < nb; ++b) {
        double e_u = e_up[base + b] - mu - h;
        double e_d = e_dn[base + b] - mu + h;
        double ep, em;
        ffeo_quasiparticle(e_u, e_d, delta * eta, &ep, &em);
        double term = ffeo_F(ep, T) + ffeo_F(em, T) + e_d + delta * delta / U[b];
        nsum_add(&tot, term);
        nsum_add(&band[b], term);
      }
    }
  }
  *omega = nsum_value(&tot);
  if (omega_band)
    for (int b = 0; b < nb; ++b) omega_band[b] = nsum_value(&band[b]);
}

/* Many (h, T, Delta) points on one set of given band energies, OpenMP over
 * points; omega_band (may be NULL) is [n][nb].  Returns the threads used. */
int ffeo_omega_given_batch(int nb, int N, const double* e_up, const double* e_dn,
                           double eta_amp, double mu, const double* U, int64_t n,
                           const double* h, const double* T, const double* delta,
                           double* omega, double* omega_band, int nthreads) {
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
    for (int64_t p = 0; p < n; ++p)
      ffeo_omega_given(nb, N, e_up, e_dn, eta_amp, mu, U, h[p], T[p], delta[p],
                       &omega[p], omega_band ? &omega_band[nb * p] : NULL);
  }
#else
  (void)nthreads;
  for (int64_t p = 0; p < n; ++p)
    ffeo_omega_given(nb, N, e_up, e_dn, eta_amp, mu, U, h[p], T[p], delta[p],
                     &omega[p], omega_band ? &omega_band[nb * p] : NULL);
#endif
  return used;
}

/* Fermi function f(E) = 1 / (1 + exp(E/T)), without overflow. */
static double fermi(double E, double T) {
  if (E >= 0.0) {
    double x = exp(-E / T);
    return x / (1.0 + x);
  }
  return 1.0 / (1.0 + exp(E / T));
}

/* Static Cooper pair susceptibility (App. C) from given band energies,
 * e_up[k*nb + e] = E_e at the spin-up momentum of k, e_dn[k*nb + e'] = E_e' at
 * the spin-down momentum, eta2[k] the squared structure factor:
 *   chi_{e e'} = -(1/N^2) sum_k eta2 G,  G = [f(-E_up) - f(E_dn)] / (0 - E_up - E_dn)
 * with E_up = e_up - mu - h, E_dn = e_dn - mu + h.  Where E_up + E_dn is below
 * 1e-7 T the quotient takes its limit, -f'(-E_up) = f(-E_up) f(E_up) / T.
 * chi[e*nb + e'] (Neumaier sums). */
void ffeo_chi_given(int nb, int N, const double* e_up, const double* e_dn,
                    const double* eta2, double mu, double h, double T, double* chi) {
  nsum acc[64];
  for (int i = 0; i < nb * nb; ++i) acc[i].s = acc[i].c = 0.0;
  const int64_t nk = (int64_t)N * N;
  for (int64_t k = 0; k < nk; ++k)
    for (int e = 0; e < nb; ++e)
      for (int f = 0; f < nb; ++f) {
        double Eu = e_up[k * nb + e] - mu - h;
        double Ed = e_dn[k * nb + f] - mu + h;
        double sum = Eu + Ed, q;
        if (fabs(sum) > 1e-7 * T)
          q = (fermi(-Eu, T) - fermi(Ed, T)) / sum; /* = -G */
        else
          q = fermi(-Eu, T) * fermi(Eu, T) / T;
        nsum_add(&acc[e * nb + f], eta2[k] * q);
      }
  for (int i = 0; i < nb * nb; ++i) chi[i] = nsum_value(&acc[i]) / (double)nk;
}

/* A batch of independent points, parallel over points with OpenMP.
 * nthreads <= 0 uses the OpenMP default.  Returns the thread count used. */
int ffeo_omega_batch(const ffeo_model* m, int64_t n, const int32_t* N,
                     const double* qx, const double* qy, const double* h,
                     const double* T, const double* delta, double* omega,
                     double* omega_band, int nthreads) {
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
    for (int64_t p = 0; p < n; ++p)
      ffeo_omega(m, N[p], qx[p], qy[p], h[p], T[p], delta[p], &omega[p],
                 omega_band ? &omega_band[2 * p] : NULL);
  }
#else
  (void)nthreads;
  for (int64_t p = 0; p < n; ++p)
    ffeo_omega(m, N[p], qx[p], qy[p], h[p], T[p], delta[p], &omega[p],
               omega_band ? &omega_band[2 * p] : NULL);
#endif
  return used;
}

/* Band energies on the whole lattice at k + Q/2: out[(j*N + i)*2 + b]. */
void ffeo_band_grid(const ffeo_model* m, int N, double qx, double qy,
                    double* out) {
  const double two_pi = 2.0 * M_PI;
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      double kx = two_pi * (double)i / (double)N;
      double ky = two_pi * (double)j / (double)N;
      ffeo_band_energies(m, kx + 0.5 * qx, ky + 0.5 * qy,
                         &out[((int64_t)j * N + i) * 2]);
    }
}

int ffeo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
