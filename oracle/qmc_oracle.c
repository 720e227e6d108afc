/*
 * Plain FP64 CPU oracle for the particle-by-particle (PbyP) electron move over a crowd of
 * walkers: Luo, Doak, Kent, "A High-Performance Design for Hierarchical Parallelism in the
 * QMCPACK Monte Carlo code" (arXiv:2209.14487), Alg. 1 lines 5-11 with the walker loop of
 * Alg. 2 (OpenMP over walkers).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file: only the
 * tests, the package's smoke check and the benchmark's CPU-baseline leg do.  It shares no
 * code, header, table or constant with the CUDA path; both are fed the same seeded inputs.
 *
 * The paper states the algorithm (Alg. 1) but not the wavefunction.  What each step
 * computes follows the standard Slater-Jastrow PbyP formulation; every reading taken where
 * the paper is silent is listed next to the function that takes it.
 *
 *   Psi(R) = det A_up(R) * det A_dn(R) * exp(-U(R))
 *   A_s[l][j] = phi_j(r_l)   (row l = l-th electron of spin s, column j = orbital j)
 *   U = sum_{i<j} u2_{s_i s_j}(r_ij) + sum_{i,I} u1(r_iI)
 *
 * Pins (tests/): cubic-polynomial reproduction and plane-wave node values of the spline,
 * central differences of value/gradient/Laplacian, Leibniz determinants, A^-1 A = I,
 * ratios against full recomputes of log|Psi|, delayed == Sherman-Morrison, the
 * free-electron zero-variance local energy, Philox known answers, Metropolis histogram;
 * DMC weights in closed form, unbiased multiplicities, the fixed-node rejection and the
 * zero-variance static population; the nonlocal term against full recomputes and the
 * exact sphere average of a plane wave (l = 0, 1, 2); the Ewald sum against the rock-salt
 * Madelung constant and its independence of the splitting.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* System description (mirrored by a ctypes Structure in oracle/__init__.py).             */
/* ------------------------------------------------------------------------------------ */
typedef struct or_system {
  int n_up, n_dn, n_orb, n_ions, grid;
  int drift;        /* r' = r + tau D(F) + sqrt(tau) chi (Metropolis-Hastings) with the     *
                     * drift D(F) of drift_vector: 1 limited, 2 D = F; 0: no drift          */
  int potential;    /* 1: add the model potential V(R) to E_L                               */
  int update;       /* 0: Sherman-Morrison; 1: delayed rank-k (Woodbury)                    */
  int delay_rank;   /* k for update == 1                                                    */
  int n_recompute;  /* generations between full recomputes; 0 = never                       */
  int j2_K, j1_K;   /* number of free radial coefficients; 0 = term absent                  */
  int analytic;     /* test mode: phi_j = single real plane wave pw_m[j], pw_kind[j]        */
  int dmc;          /* 1: fixed node (DMC): a move that changes the determinant's sign is   *
                     * rejected                                                             */
  double L, tau, j2_rc, j1_rc;
  uint64_t seed;
  const double* table;  /* [G][G][G][n_orb] periodic cubic B-spline coefficients */
  const double* ions;   /* [n_ions][3]                                           */
  const double* j2_uu;  /* [j2_K] like-spin pair functor                         */
  const double* j2_ud;  /* [j2_K] unlike-spin pair functor                       */
  const double* j1;     /* [j1_K] electron-ion functor                           */
  const int* pw_m;      /* [n_orb][3] integer wave vectors (analytic mode)       */
  const int* pw_kind;   /* [n_orb]: 0 constant, 1 cos, 2 sin (analytic mode)     */
  int nl_n, nl_pad;     /* nonlocal channels l = 0..nl_n-1 (0: none), at most 3    */
  double nl_rc;         /* their cutoff radius                                    */
  double nl_a[3];       /* v_l(r) = nl_a[l] exp(-(r / nl_s[l])^2), r < nl_rc       */
  double nl_s[3];
  int coul;             /* 1: add the Ewald Coulomb energy (electrons -1, ions +Z) */
  int coul_mmax;        /* reciprocal vectors k = 2 pi m / L with |m|^2 <= mmax^2  */
  double coul_alpha;    /* Ewald splitting parameter                              */
  double coul_Z;        /* ion charge                                             */
} or_system;

static const double OR_TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------------------ */
/* Counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4).         */
/* Round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2; c = (hi1^c1^k0, lo1, hi0^c3^k1, lo0);     */
/* the key is bumped by the Weyl constants between rounds.                               */
/* ------------------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in (0, 1]: u = (k + 1/2) 2^-53 with k = (a >> 5) 2^26 + (b >> 6). */
static double u53(uint32_t a, uint32_t b) {
  uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return ((double)k + 0.5) * 0x1p-53;
}

/* Random numbers of one proposal (Alg. 1 line 5, "delta"), read as a Gaussian step.
 * key = (low 32 bits of seed, walker ^ high 32 bits of seed)
 * counter = (generation, electron, slot, 0): slot 0 -> chi_x, chi_y (Box-Muller of two
 * uniforms), slot 1 -> chi_z, slot 2 -> the acceptance uniform. */
void or_move_draws(uint64_t seed, uint32_t walker, uint32_t gen, uint32_t iel, double* chi,
                   double* uacc) {
  uint32_t key[2] = {(uint32_t)seed, walker ^ (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {gen, iel, 0u, 0u};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  double u1 = u53(x[0], x[1]), u2 = u53(x[2], x[3]);
  double rad = sqrt(-2.0 * log(u1));
  chi[0] = rad * cos(OR_TWO_PI * u2);
  chi[1] = rad * sin(OR_TWO_PI * u2);
  ctr[2] = 1u;
  or_philox4x32_10(ctr, key, x);
  double u3 = u53(x[0], x[1]), u4 = u53(x[2], x[3]);
  chi[2] = sqrt(-2.0 * log(u3)) * cos(OR_TWO_PI * u4);
  ctr[2] = 2u;
  or_philox4x32_10(ctr, key, x);
  *uacc = u53(x[0], x[1]);
}

/* ------------------------------------------------------------------------------------ */
/* Uniform cubic B-spline basis on one cell, t in [0,1]: weights of the 4 coefficients   */
/* that touch the cell, and their first and second derivatives in t.                     */
/* ------------------------------------------------------------------------------------ */
static void cubic_basis(double t, double* b, double* db, double* d2b) {
  double t2 = t * t, t3 = t2 * t, s = 1.0 - t;
  b[0] = s * s * s / 6.0;
  b[1] = (3.0 * t3 - 6.0 * t2 + 4.0) / 6.0;
  b[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) / 6.0;
  b[3] = t3 / 6.0;
  db[0] = -0.5 * s * s;
  db[1] = 1.5 * t2 - 2.0 * t;
  db[2] = -1.5 * t2 + t + 0.5;
  db[3] = 0.5 * t2;
  d2b[0] = s;
  d2b[1] = 3.0 * t - 2.0;
  d2b[2] = -3.0 * t + 1.0;
  d2b[3] = t;
}

/* Radial functor u(r) (one- and two-body Jastrow), reading: K free coefficients followed
 * by three zeros, knot spacing h = rc/K; for r < rc, i = floor(r/h) (at most K-1),
 * t = r/h - i, u = sum_m c_{i+m} b_m(t); u = 0 for r >= rc (strict cutoff). */
void or_radial(const double* c, int K, double rc, double r, double* out) {
  out[0] = out[1] = out[2] = 0.0;
  if (!(r < rc)) return;
  double h = rc / K;
  double x = r / h;
  int i = (int)floor(x);
  if (i > K - 1) i = K - 1;
  if (i < 0) i = 0;
  double t = x - i;
  double b[4], db[4], d2b[4];
  cubic_basis(t, b, db, d2b);
  for (int m = 0; m < 4; ++m) {
    double cm = (i + m < K) ? c[i + m] : 0.0;
    out[0] += cm * b[m];
    out[1] += cm * db[m] / h;
    out[2] += cm * d2b[m] / (h * h);
  }
}

static double wrap1(double x, double L) { return x - L * floor(x / L); }

/* Minimum-image displacement a - b and its length (round to nearest, ties to even). */
static double min_image(const double* a, const double* b, double L, double* d) {
  double r2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    double x = a[k] - b[k];
    x -= L * nearbyint(x / L);
    d[k] = x;
    r2 += x * x;
  }
  return sqrt(r2);
}

/* ------------------------------------------------------------------------------------ */
/* Orbitals: phi_j, grad phi_j, lap phi_j at r (Alg. 1 lines 7-8: the vector loop over    */
/* orbitals).  Tricubic B-spline on a periodic G^3 grid, reading: cell g (g = floor(s),   */
/* s = r G / L, at most G-1) combines coefficients g-1..g+2 in each direction.            */
/* ------------------------------------------------------------------------------------ */
static void analytic_wave(const or_system* s, const double* r, int n, double* v, double* g,
                          double* l) {
  double k0 = OR_TWO_PI / s->L;
  for (int j = 0; j < n; ++j) {
    const int* m = s->pw_m + 3 * j;
    double k[3] = {k0 * m[0], k0 * m[1], k0 * m[2]};
    double ph = k[0] * r[0] + k[1] * r[1] + k[2] * r[2];
    double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    int kind = s->pw_kind[j];
    double val, dval; /* w and dw/dph */
    if (kind == 0) { val = 1.0; dval = 0.0; }
    else if (kind == 1) { val = cos(ph); dval = -sin(ph); }
    else { val = sin(ph); dval = cos(ph); }
    v[j] = val;
    for (int d = 0; d < 3; ++d) g[3 * j + d] = k[d] * dval;
    l[j] = -kk * val;
  }
}

void or_spo_vgl(const or_system* s, const double* r_in, int n, double* v, double* g,
                double* l) {
  double r[3] = {wrap1(r_in[0], s->L), wrap1(r_in[1], s->L), wrap1(r_in[2], s->L)};
  if (s->analytic) {
    analytic_wave(s, r, n, v, g, l);
    return;
  }
  int G = s->grid;
  double dinv = (double)G / s->L;
  int cell[3];
  double b[3][4], db[3][4], d2b[3][4];
  for (int d = 0; d < 3; ++d) {
    double x = r[d] * dinv;
    int ig = (int)floor(x);
    if (ig > G - 1) ig = G - 1;
    if (ig < 0) ig = 0;
    cell[d] = ig;
    cubic_basis(x - ig, b[d], db[d], d2b[d]);
  }
  for (int j = 0; j < n; ++j) {
    v[j] = 0.0;
    g[3 * j] = g[3 * j + 1] = g[3 * j + 2] = 0.0;
    l[j] = 0.0;
  }
  for (int a = 0; a < 4; ++a) {
    int ix = ((cell[0] - 1 + a) % G + G) % G;
    for (int bb = 0; bb < 4; ++bb) {
      int iy = ((cell[1] - 1 + bb) % G + G) % G;
      for (int c = 0; c < 4; ++c) {
        int iz = ((cell[2] - 1 + c) % G + G) % G;
        const double* row = s->table + (((size_t)ix * G + iy) * G + iz) * (size_t)s->n_orb;
        double wv = b[0][a] * b[1][bb] * b[2][c];
        double wx = db[0][a] * b[1][bb] * b[2][c] * dinv;
        double wy = b[0][a] * db[1][bb] * b[2][c] * dinv;
        double wz = b[0][a] * b[1][bb] * db[2][c] * dinv;
        double wl = (d2b[0][a] * b[1][bb] * b[2][c] + b[0][a] * d2b[1][bb] * b[2][c] +
                     b[0][a] * b[1][bb] * d2b[2][c]) * dinv * dinv;
        for (int j = 0; j < n; ++j) {
          double cf = row[j];
          v[j] += wv * cf;
          g[3 * j] += wx * cf;
          g[3 * j + 1] += wy * cf;
          g[3 * j + 2] += wz * cf;
          l[j] += wl * cf;
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Jastrow pieces.                                                                       */
/* ------------------------------------------------------------------------------------ */
static int n_el(const or_system* s) { return s->n_up + s->n_dn; }
static int spin_of(const or_system* s, int i) { return i < s->n_up ? 0 : 1; }

static const double* pair_coefs(const or_system* s, int i, int j) {
  return spin_of(s, i) == spin_of(s, j) ? s->j2_uu : s->j2_ud;
}

/* U_i(r) = sum_{j != i} u2(|r - r_j|) + sum_I u1(|r - R_I|), with its gradient in r and
 * its Laplacian (u'' + 2u'/r per term).  Electron i's own position is skipped. */
static void jastrow_one(const or_system* s, const double* R, int i, const double* r,
                        double* U, double* grad, double* lap) {
  *U = 0.0;
  grad[0] = grad[1] = grad[2] = 0.0;
  *lap = 0.0;
  int N = n_el(s);
  double d[3], f[3];
  if (s->j2_K > 0) {
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double rr = min_image(r, R + 3 * j, s->L, d);
      or_radial(pair_coefs(s, i, j), s->j2_K, s->j2_rc, rr, f);
      *U += f[0];
      if (rr > 0.0) {
        for (int k = 0; k < 3; ++k) grad[k] += f[1] * d[k] / rr;
        *lap += f[2] + 2.0 * f[1] / rr;
      }
    }
  }
  if (s->j1_K > 0) {
    for (int I = 0; I < s->n_ions; ++I) {
      double rr = min_image(r, s->ions + 3 * I, s->L, d);
      or_radial(s->j1, s->j1_K, s->j1_rc, rr, f);
      *U += f[0];
      if (rr > 0.0) {
        for (int k = 0; k < 3; ++k) grad[k] += f[1] * d[k] / rr;
        *lap += f[2] + 2.0 * f[1] / rr;
      }
    }
  }
}

/* U(R) by its definition: pairs i<j and electron-ion terms. */
double or_jastrow_U(const or_system* s, const double* R) {
  int N = n_el(s);
  double U = 0.0, d[3], f[3];
  if (s->j2_K > 0)
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j) {
        double rr = min_image(R + 3 * i, R + 3 * j, s->L, d);
        or_radial(pair_coefs(s, i, j), s->j2_K, s->j2_rc, rr, f);
        U += f[0];
      }
  if (s->j1_K > 0)
    for (int i = 0; i < N; ++i)
      for (int I = 0; I < s->n_ions; ++I) {
        double rr = min_image(R + 3 * i, s->ions + 3 * I, s->L, d);
        or_radial(s->j1, s->j1_K, s->j1_rc, rr, f);
        U += f[0];
      }
  return U;
}

/* Model potential, reading (the paper gives no Hamiltonian): smooth Gaussians,
 * v_ee = exp(-r^2), v_eI = -2 exp(-r^2/2), minimum image, zero for r >= L/2. */
double or_coulomb(const or_system* s, const double* R, int images);

double or_potential(const or_system* s, const double* R) {
  double Vc = s->coul ? or_coulomb(s, R, 0) : 0.0;
  if (!s->potential) return Vc;
  int N = n_el(s);
  double V = 0.0, d[3], half = 0.5 * s->L;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      double rr = min_image(R + 3 * i, R + 3 * j, s->L, d);
      if (rr < half) V += exp(-rr * rr);
    }
  for (int i = 0; i < N; ++i)
    for (int I = 0; I < s->n_ions; ++I) {
      double rr = min_image(R + 3 * i, s->ions + 3 * I, s->L, d);
      if (rr < half) V += -2.0 * exp(-0.5 * rr * rr);
    }
  return V + Vc;
}

/* ------------------------------------------------------------------------------------ */
/* Coulomb energy by Ewald summation, reading (the paper's runs use it; its text gives no */
/* form): charges -1 (electrons) and +Z (ions) in the periodic cube, V = L^3,             */
/*   E = sum_{a<b} q_a q_b erfc(alpha r_ab) / r_ab                      (real space)      */
/*     + (2 pi / V) sum_{k != 0} exp(-k^2 / (4 alpha^2)) / k^2 |S(k)|^2 (reciprocal)      */
/*     - (alpha / sqrt(pi)) sum_a q_a^2 - pi Q^2 / (2 V alpha^2)        (self, background)*/
/* S(k) = sum_a q_a exp(i k.r_a), k = 2 pi m / L over integer m with 0 < |m|^2 <= mmax^2,  */
/* Q = sum_a q_a.  The real-space sum takes the minimum image of each pair (images = 0)   */
/* or every pair and self-image within the 27 nearest cells (images = 1).                */
/* ------------------------------------------------------------------------------------ */
double or_coulomb(const or_system* s, const double* R, int images) {
  const int N = n_el(s), NI = s->n_ions, M = N + NI;
  const double L = s->L, V = L * L * L, a = s->coul_alpha, Z = s->coul_Z;
  double* x = (double*)malloc(sizeof(double) * 3 * (M > 0 ? M : 1));
  double* q = (double*)malloc(sizeof(double) * (M > 0 ? M : 1));
  for (int i = 0; i < N; ++i) {
    for (int k = 0; k < 3; ++k) x[3 * i + k] = R[3 * i + k];
    q[i] = -1.0;
  }
  for (int I = 0; I < NI; ++I) {
    for (int k = 0; k < 3; ++k) x[3 * (N + I) + k] = s->ions[3 * I + k];
    q[N + I] = Z;
  }
  double Ereal = 0.0, Erec = 0.0, Q = 0.0, Q2 = 0.0;
  for (int i = 0; i < M; ++i) {
    Q += q[i];
    Q2 += q[i] * q[i];
  }
  for (int i = 0; i < M; ++i)
    for (int j = i; j < M; ++j) {
      double d[3];
      if (!images) {
        if (j == i) continue;
        double r = min_image(x + 3 * i, x + 3 * j, L, d);
        Ereal += q[i] * q[j] * erfc(a * r) / r;
        continue;
      }
      for (int k = 0; k < 3; ++k) d[k] = x[3 * i + k] - x[3 * j + k];
      for (int n0 = -1; n0 <= 1; ++n0)
        for (int n1 = -1; n1 <= 1; ++n1)
          for (int n2 = -1; n2 <= 1; ++n2) {
            if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;
            double e0 = d[0] + n0 * L, e1 = d[1] + n1 * L, e2 = d[2] + n2 * L;
            double r = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
            /* a pair's images once each; a self-image pair (n, -n) twice, so halve it */
            Ereal += (i == j ? 0.5 : 1.0) * q[i] * q[j] * erfc(a * r) / r;
          }
    }
  const int mm = s->coul_mmax;
  for (int m0 = -mm; m0 <= mm; ++m0)
    for (int m1 = -mm; m1 <= mm; ++m1)
      for (int m2 = -mm; m2 <= mm; ++m2) {
        int m2s = m0 * m0 + m1 * m1 + m2 * m2;
        if (m2s == 0 || m2s > mm * mm) continue;
        double k[3] = {OR_TWO_PI * m0 / L, OR_TWO_PI * m1 / L, OR_TWO_PI * m2 / L};
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double re = 0.0, im = 0.0;
        for (int i = 0; i < M; ++i) {
          double ph = k[0] * x[3 * i] + k[1] * x[3 * i + 1] + k[2] * x[3 * i + 2];
          re += q[i] * cos(ph);
          im += q[i] * sin(ph);
        }
        Erec += exp(-k2 / (4.0 * a * a)) / k2 * (re * re + im * im);
      }
  Erec *= OR_TWO_PI / V;
  free(x);
  free(q);
  const double sqrt_pi = 1.7724538509055160273;
  return Ereal + Erec - a / sqrt_pi * Q2 - 0.5 * OR_TWO_PI * Q * Q / (2.0 * V * a * a);
}

/* ------------------------------------------------------------------------------------ */
/* Dense linear algebra: LU with partial pivoting (row exchanges).                       */
/* ------------------------------------------------------------------------------------ */
static int lu_factor(double* a, int n, int* piv, double* logabs, int* sign) {
  *logabs = 0.0;
  *sign = 1;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return 1;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t;
      }
      *sign = -*sign;
    }
    double akk = a[k * n + k];
    if (akk < 0.0) *sign = -*sign;
    *logabs += log(fabs(akk));
    for (int i = k + 1; i < n; ++i) {
      double lik = a[i * n + k] / akk;
      a[i * n + k] = lik;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= lik * a[k * n + j];
    }
  }
  return 0;
}

static void lu_solve(const double* lu, const int* piv, int n, double* x) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= lu[i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= lu[i * n + j] * x[j];
    x[i] /= lu[i * n + i];
  }
}

/* log|det a| and its sign; returns 1 for an exactly singular matrix. */
int or_det(const double* a, int n, double* logabs, int* sign) {
  if (n == 0) { *logabs = 0.0; *sign = 1; return 0; }
  double* w = (double*)malloc(sizeof(double) * n * n);
  int* piv = (int*)malloc(sizeof(int) * n);
  memcpy(w, a, sizeof(double) * n * n);
  int st = lu_factor(w, n, piv, logabs, sign);
  free(w); free(piv);
  return st;
}

/* inv = a^-1 column by column from the LU factors; returns 1 if singular. */
int or_inverse(const double* a, int n, double* inv, double* logabs, int* sign) {
  if (n == 0) { *logabs = 0.0; *sign = 1; return 0; }
  double* w = (double*)malloc(sizeof(double) * n * n);
  double* col = (double*)malloc(sizeof(double) * n);
  int* piv = (int*)malloc(sizeof(int) * n);
  memcpy(w, a, sizeof(double) * n * n);
  int st = lu_factor(w, n, piv, logabs, sign);
  if (st == 0) {
    for (int c = 0; c < n; ++c) {
      for (int i = 0; i < n; ++i) col[i] = (i == c) ? 1.0 : 0.0;
      lu_solve(w, piv, n, col);
      for (int i = 0; i < n; ++i) inv[i * n + c] = col[i];
    }
  }
  free(w); free(col); free(piv);
  return st;
}

/* ------------------------------------------------------------------------------------ */
/* Whole-configuration quantities by their definitions (full recomputes).                */
/* ------------------------------------------------------------------------------------ */
static int spin_size(const or_system* s, int sp) { return sp == 0 ? s->n_up : s->n_dn; }
static int spin_off(const or_system* s, int sp) { return sp == 0 ? 0 : s->n_up; }

/* Fills A, dA (3 per entry), d2A of one spin block from the positions. */
static void build_rows(const or_system* s, const double* R, int sp, double* A, double* dA,
                       double* d2A) {
  int ns = spin_size(s, sp), off = spin_off(s, sp);
  for (int l = 0; l < ns; ++l)
    or_spo_vgl(s, R + 3 * (off + l), ns, A + (size_t)l * ns, dA + (size_t)l * ns * 3,
               d2A + (size_t)l * ns);
}

/* log|Psi| and sign(Psi) = log|det A_up| + log|det A_dn| - U; returns 1 if singular. */
int or_logpsi(const or_system* s, const double* R, double* logabs, int* sign) {
  *logabs = 0.0;
  *sign = 1;
  for (int sp = 0; sp < 2; ++sp) {
    int ns = spin_size(s, sp);
    if (ns == 0) continue;
    double* A = (double*)malloc(sizeof(double) * ns * ns);
    double* dA = (double*)malloc(sizeof(double) * ns * ns * 3);
    double* d2A = (double*)malloc(sizeof(double) * ns * ns);
    build_rows(s, R, sp, A, dA, d2A);
    double la; int sg;
    int st = or_det(A, ns, &la, &sg);
    free(A); free(dA); free(d2A);
    if (st) return 1;
    *logabs += la;
    *sign *= sg;
  }
  *logabs -= or_jastrow_U(s, R);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Nonlocal pseudopotential, reading (the paper's NiO runs use pseudopotentials; its text */
/* gives no form): every ion carries channels l = 0..nl_n-1, v_l(r) = a_l exp(-(r/s_l)^2) */
/* for r < nl_rc, zero beyond (minimum image).  For electron i at d = r_i - R_I, r = |d|: */
/*   V_iI = sum_l v_l(r) (2l+1) (1/12) sum_q P_l(d.u_q / r) Psi(r_i -> R_I + r u_q)/Psi(R) */
/* with u_q the 12 vertices of an icosahedron in a fixed orientation (a spherical design  */
/* that integrates polynomials of degree <= 5 exactly), P_0 = 1, P_1 = x,                 */
/* P_2 = (3x^2 - 1)/2.  E_L gains sum_{i,I} V_iI (the locality approximation).            */
/* ------------------------------------------------------------------------------------ */
static void icosahedron(double u[12][3]) {
  const double ph = 0.5 * (1.0 + sqrt(5.0)), nrm = 1.0 / sqrt(1.0 + ph * ph);
  const double sg[4][2] = {{1, 1}, {-1, 1}, {1, -1}, {-1, -1}};
  for (int k = 0; k < 4; ++k) {  /* (0, +-1, +-phi) and its two cyclic shifts */
    double a = sg[k][0] * nrm, b = sg[k][1] * ph * nrm;
    u[k][0] = 0.0;    u[k][1] = a;        u[k][2] = b;
    u[4 + k][0] = a;  u[4 + k][1] = b;    u[4 + k][2] = 0.0;
    u[8 + k][0] = b;  u[8 + k][1] = 0.0;  u[8 + k][2] = a;
  }
}

static double legendre(int l, double x) {
  return l == 0 ? 1.0 : (l == 1 ? x : 1.5 * x * x - 0.5);
}

/* Psi(R with r_i -> rp) / Psi(R) from two full recomputes. */
static double ratio_direct(const or_system* s, const double* R, int i, const double* rp) {
  int N = n_el(s);
  double* R2 = (double*)malloc(sizeof(double) * 3 * N);
  memcpy(R2, R, sizeof(double) * 3 * N);
  for (int k = 0; k < 3; ++k) R2[3 * i + k] = rp[k];
  double la0, la1;
  int s0, s1;
  int bad = or_logpsi(s, R, &la0, &s0) || or_logpsi(s, R2, &la1, &s1);
  free(R2);
  return bad ? NAN : (double)(s0 * s1) * exp(la1 - la0);
}

/* The same ratio from electron i's column of A^-1 (one row of A replaced):
 * phi(rp) . Ainv[:, l] times exp(-(U_i(rp) - U_i(r_i))). */
static double ratio_column(const or_system* s, const double* R, int i, const double* rp,
                           const double* Binv) {
  int sp = spin_of(s, i), ns = spin_size(s, sp), l = i - spin_off(s, sp);
  double* v = (double*)malloc(sizeof(double) * ns * 5);
  or_spo_vgl(s, rp, ns, v, v + ns, v + 4 * ns);
  double det = 0.0;
  for (int j = 0; j < ns; ++j) det += v[j] * Binv[(size_t)j * ns + l];
  free(v);
  double U0, U1, gU[3], lU;
  jastrow_one(s, R, i, R + 3 * i, &U0, gU, &lU);
  jastrow_one(s, R, i, rp, &U1, gU, &lU);
  return det * exp(-(U1 - U0));
}

/* sum_{i,I} V_iI; Binv[sp] = A_sp^-1 (row-major), or NULL for the direct ratios. */
static double nlpp_energy(const or_system* s, const double* R, const double* const* Binv) {
  if (s->nl_n <= 0 || s->n_ions == 0) return 0.0;
  double u[12][3];
  icosahedron(u);
  int N = n_el(s);
  double V = 0.0;
  for (int i = 0; i < N; ++i)
    for (int I = 0; I < s->n_ions; ++I) {
      double d[3];
      double r = min_image(R + 3 * i, s->ions + 3 * I, s->L, d);
      if (!(r < s->nl_rc) || r == 0.0) continue;
      double acc[3] = {0.0, 0.0, 0.0};
      for (int q = 0; q < 12; ++q) {
        double rp[3], c = 0.0;
        for (int k = 0; k < 3; ++k) {
          rp[k] = R[3 * i + k] - d[k] + r * u[q][k];  /* the ion's image + r u_q */
          c += d[k] * u[q][k];
        }
        c /= r;
        double rho = Binv ? ratio_column(s, R, i, rp, Binv[spin_of(s, i)])
                          : ratio_direct(s, R, i, rp);
        for (int l = 0; l < s->nl_n; ++l) acc[l] += legendre(l, c) * rho;
      }
      for (int l = 0; l < s->nl_n; ++l) {
        double x = r / s->nl_s[l];
        V += s->nl_a[l] * exp(-x * x) * (double)(2 * l + 1) * acc[l] / 12.0;
      }
    }
  return V;
}

/* grad_i log Psi and lap_i log Psi for every electron, and the local energy
 * E_L = -1/2 sum_i [lap_i log Psi + |grad_i log Psi|^2] + V  (Alg. 1 line 11), with
 * grad_i log D = sum_j dA[l][j] Ainv[j][l],  lap_i D / D = sum_j d2A[l][j] Ainv[j][l]. */
int or_local_energy(const or_system* s, const double* R, double* grad, double* lap,
                    double* eloc) {
  int N = n_el(s);
  double kin = 0.0;
  double* Bk[2] = {NULL, NULL};
  for (int sp = 0; sp < 2; ++sp) {
    int ns = spin_size(s, sp), off = spin_off(s, sp);
    if (ns == 0) continue;
    double* A = (double*)malloc(sizeof(double) * ns * ns);
    double* dA = (double*)malloc(sizeof(double) * ns * ns * 3);
    double* d2A = (double*)malloc(sizeof(double) * ns * ns);
    double* B = (double*)malloc(sizeof(double) * ns * ns);
    Bk[sp] = B;
    build_rows(s, R, sp, A, dA, d2A);
    double la; int sg;
    if (or_inverse(A, ns, B, &la, &sg)) {
      free(A); free(dA); free(d2A); free(Bk[0]); free(Bk[1]);
      return 1;
    }
    for (int l = 0; l < ns; ++l) {
      int i = off + l;
      double gD[3] = {0, 0, 0}, lD = 0.0;
      for (int j = 0; j < ns; ++j) {
        double bji = B[j * ns + l];
        for (int k = 0; k < 3; ++k) gD[k] += dA[((size_t)l * ns + j) * 3 + k] * bji;
        lD += d2A[(size_t)l * ns + j] * bji;
      }
      double U, gU[3], lU;
      jastrow_one(s, R, i, R + 3 * i, &U, gU, &lU);
      double g[3], g2 = 0.0, gD2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        g[k] = gD[k] - gU[k];
        g2 += g[k] * g[k];
        gD2 += gD[k] * gD[k];
      }
      double lp = (lD - gD2) - lU;
      if (grad) for (int k = 0; k < 3; ++k) grad[3 * i + k] = g[k];
      if (lap) lap[i] = lp;
      kin += -0.5 * (lp + g2);
    }
    free(A); free(dA); free(d2A);
  }
  (void)N;
  if (eloc) *eloc = kin + or_potential(s, R) + nlpp_energy(s, R, (const double* const*)Bk);
  free(Bk[0]); free(Bk[1]);
  return 0;
}

/* The nonlocal term by its plain definition: every ratio from two full recomputes of
 * log|Psi| (direct = 1), or from the inverses of a full recompute (direct = 0).  NaN if
 * a Slater matrix is singular. */
double or_nlpp(const or_system* s, const double* R, int direct) {
  if (direct) return nlpp_energy(s, R, NULL);
  double* Bk[2] = {NULL, NULL};
  double out = 0.0;
  for (int sp = 0; sp < 2 && !isnan(out); ++sp) {
    int ns = spin_size(s, sp);
    if (ns == 0) continue;
    double* A = (double*)malloc(sizeof(double) * ns * ns);
    double* dA = (double*)malloc(sizeof(double) * ns * ns * 3);
    double* d2A = (double*)malloc(sizeof(double) * ns * ns);
    Bk[sp] = (double*)malloc(sizeof(double) * ns * ns);
    build_rows(s, R, sp, A, dA, d2A);
    double la; int sg;
    if (or_inverse(A, ns, Bk[sp], &la, &sg)) out = NAN;
    free(A); free(dA); free(d2A);
  }
  if (!isnan(out)) out = nlpp_energy(s, R, (const double* const*)Bk);
  free(Bk[0]); free(Bk[1]);
  return out;
}

/* ------------------------------------------------------------------------------------ */
/* Crowd: W walkers moved particle by particle (Alg. 1 lines 4-9), fine-grained calls    */
/* mirror the batched API (propose / accept / local energy) for parity checks.           */
/* ------------------------------------------------------------------------------------ */
typedef struct or_walker {
  double* A[2];    /* [n][n]    A[l][j] = phi_j(r_l)           */
  double* dA[2];   /* [n][n][3]                                 */
  double* d2A[2];  /* [n][n]                                    */
  double* B[2];    /* [n][n]    B = A^-1 at the window start    */
  double logdet[2];
  int sign[2];
  /* delayed window: rows p_a replaced, V[a] = phi' - (row p_a before it) */
  int m[2];
  int* P[2];       /* [k] */
  double* V[2];    /* [k][n] */
  /* pending proposal */
  int pend_iel;
  double rp[3], disp[3], F[3], Fp[3];
  double rhoD, rho, dU, logGf;
  double *pv, *pg, *pl;  /* phi', grad phi', lap phi' at r' */
  double* col;           /* current inverse column of the moving row */
  int valid;
} or_walker;

typedef struct or_crowd {
  or_system s;
  int W, N, nmax;
  uint32_t gen;
  double* R;  /* [W][N][3] */
  or_walker* wk;
} or_crowd;

static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

static void walker_free(or_walker* w) {
  for (int sp = 0; sp < 2; ++sp) {
    free(w->A[sp]); free(w->dA[sp]); free(w->d2A[sp]); free(w->B[sp]);
    free(w->P[sp]); free(w->V[sp]);
  }
  free(w->pv); free(w->pg); free(w->pl); free(w->col);
}

/* Builds A, dA, d2A from the positions and B = A^-1 by LU; discards any delayed window. */
static int walker_recompute(or_crowd* c, int w) {
  const or_system* s = &c->s;
  or_walker* wk = &c->wk[w];
  double* R = c->R + (size_t)w * c->N * 3;
  int st = 0;
  for (int sp = 0; sp < 2; ++sp) {
    int ns = spin_size(s, sp);
    wk->m[sp] = 0;
    if (ns == 0) { wk->logdet[sp] = 0.0; wk->sign[sp] = 1; continue; }
    build_rows(s, R, sp, wk->A[sp], wk->dA[sp], wk->d2A[sp]);
    if (or_inverse(wk->A[sp], ns, wk->B[sp], &wk->logdet[sp], &wk->sign[sp])) st = 1;
  }
  return st;
}

or_crowd* or_crowd_create(const or_system* s, int W, const double* R) {
  or_crowd* c = (or_crowd*)calloc(1, sizeof(or_crowd));
  c->s = *s;
  c->W = W;
  c->N = n_el(s);
  c->nmax = s->n_up > s->n_dn ? s->n_up : s->n_dn;
  c->R = dalloc((size_t)W * c->N * 3);
  memcpy(c->R, R, sizeof(double) * W * c->N * 3);
  c->wk = (or_walker*)calloc(W, sizeof(or_walker));
  int k = s->delay_rank > 0 ? s->delay_rank : 1;
  for (int w = 0; w < W; ++w) {
    or_walker* wk = &c->wk[w];
    for (int sp = 0; sp < 2; ++sp) {
      size_t n = (size_t)spin_size(s, sp);
      wk->A[sp] = dalloc(n * n);
      wk->dA[sp] = dalloc(n * n * 3);
      wk->d2A[sp] = dalloc(n * n);
      wk->B[sp] = dalloc(n * n);
      wk->P[sp] = (int*)calloc(k, sizeof(int));
      wk->V[sp] = dalloc((size_t)k * n);
    }
    wk->pv = dalloc(c->nmax);
    wk->pg = dalloc((size_t)c->nmax * 3);
    wk->pl = dalloc(c->nmax);
    wk->col = dalloc(c->nmax);
    wk->pend_iel = -1;
  }
  return c;
}

void or_crowd_destroy(or_crowd* c) {
  if (!c) return;
  for (int w = 0; w < c->W; ++w) walker_free(&c->wk[w]);
  free(c->wk);
  free(c->R);
  free(c);
}

int or_crowd_recompute(or_crowd* c) {
  int st = 0;
  for (int w = 0; w < c->W; ++w) st |= walker_recompute(c, w);
  return st;
}

/* S = I_m + V B P (m x m) of a delayed window. */
static void window_S(const or_walker* wk, int sp, int ns, double* S) {
  int m = wk->m[sp];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      double acc = (a == b) ? 1.0 : 0.0;
      for (int j = 0; j < ns; ++j) acc += wk->V[sp][a * ns + j] * wk->B[sp][j * ns + wk->P[sp][b]];
      S[a * m + b] = acc;
    }
}

/* Column p of the current inverse.  Sherman-Morrison: B[:,p].  Delayed window
 * (A_cur = A_0 + P V): Ainv_cur[:,p] = B[:,p] - (B P) S^-1 (V B[:,p]). */
static void current_column(const or_crowd* c, const or_walker* wk, int sp, int p, double* col) {
  int ns = spin_size(&c->s, sp);
  for (int j = 0; j < ns; ++j) col[j] = wk->B[sp][j * ns + p];
  int m = wk->m[sp];
  if (m == 0) return;
  double* S = dalloc((size_t)m * m);
  double* y = dalloc(m);
  int* piv = (int*)calloc(m, sizeof(int));
  window_S(wk, sp, ns, S);
  for (int a = 0; a < m; ++a) {
    double acc = 0.0;
    for (int j = 0; j < ns; ++j) acc += wk->V[sp][a * ns + j] * wk->B[sp][j * ns + p];
    y[a] = acc;
  }
  double la; int sg;
  lu_factor(S, m, piv, &la, &sg);
  lu_solve(S, piv, m, y);
  for (int j = 0; j < ns; ++j) {
    double acc = 0.0;
    for (int b = 0; b < m; ++b) acc += wk->B[sp][j * ns + wk->P[sp][b]] * y[b];
    col[j] -= acc;
  }
  free(S); free(y); free(piv);
}

/* Applies a delayed window: B <- B - (B P) S^-1 (V B), then empties it. */
static void window_flush(const or_crowd* c, or_walker* wk, int sp) {
  int m = wk->m[sp];
  if (m == 0) return;
  int ns = spin_size(&c->s, sp);
  double* S = dalloc((size_t)m * m);
  double* Y = dalloc((size_t)m * ns);
  double* BP = dalloc((size_t)ns * m);
  double* col = dalloc(m);
  int* piv = (int*)calloc(m, sizeof(int));
  window_S(wk, sp, ns, S);
  for (int a = 0; a < m; ++a)
    for (int l = 0; l < ns; ++l) {
      double acc = 0.0;
      for (int j = 0; j < ns; ++j) acc += wk->V[sp][a * ns + j] * wk->B[sp][j * ns + l];
      Y[a * ns + l] = acc;
    }
  for (int j = 0; j < ns; ++j)
    for (int b = 0; b < m; ++b) BP[j * m + b] = wk->B[sp][j * ns + wk->P[sp][b]];
  double la; int sg;
  lu_factor(S, m, piv, &la, &sg);
  for (int l = 0; l < ns; ++l) { /* Z[:,l] = S^-1 Y[:,l] */
    for (int a = 0; a < m; ++a) col[a] = Y[a * ns + l];
    lu_solve(S, piv, m, col);
    for (int a = 0; a < m; ++a) Y[a * ns + l] = col[a];
  }
  for (int j = 0; j < ns; ++j)
    for (int l = 0; l < ns; ++l) {
      double acc = 0.0;
      for (int b = 0; b < m; ++b) acc += BP[j * m + b] * Y[b * ns + l];
      wk->B[sp][j * ns + l] -= acc;
    }
  wk->m[sp] = 0;
  free(S); free(Y); free(BP); free(col); free(piv);
}

void or_crowd_flush(or_crowd* c) {
  for (int w = 0; w < c->W; ++w)
    for (int sp = 0; sp < 2; ++sp) window_flush(c, &c->wk[w], sp);
}

/* grad_i log Psi at the current positions (the drift of Alg. 1 line 5). */
static void walker_grad(const or_crowd* c, or_walker* wk, int w, int i, double* F) {
  const or_system* s = &c->s;
  int sp = spin_of(s, i), p = i - spin_off(s, sp), ns = spin_size(s, sp);
  const double* R = c->R + (size_t)w * c->N * 3;
  current_column(c, wk, sp, p, wk->col);
  double gD[3] = {0, 0, 0};
  for (int j = 0; j < ns; ++j)
    for (int k = 0; k < 3; ++k) gD[k] += wk->dA[sp][((size_t)p * ns + j) * 3 + k] * wk->col[j];
  double U, gU[3], lU;
  jastrow_one(s, R, i, R + 3 * i, &U, gU, &lU);
  for (int k = 0; k < 3; ++k) F[k] = gD[k] - gU[k];
}

/* Ratio Psi(R')/Psi(R) and grad_i log Psi(R') for electron i moved to rp (Alg. 1 lines
 * 7-8).  Stores the proposal for a following accept. */
static void walker_ratio_grad(const or_crowd* c, or_walker* wk, int w, int i, const double* rp_in) {
  const or_system* s = &c->s;
  int sp = spin_of(s, i), p = i - spin_off(s, sp), ns = spin_size(s, sp);
  const double* R = c->R + (size_t)w * c->N * 3;
  double rp[3] = {wrap1(rp_in[0], s->L), wrap1(rp_in[1], s->L), wrap1(rp_in[2], s->L)};
  for (int k = 0; k < 3; ++k) wk->rp[k] = rp[k];
  current_column(c, wk, sp, p, wk->col);
  or_spo_vgl(s, rp, ns, wk->pv, wk->pg, wk->pl);
  double rhoD = 0.0, gD[3] = {0, 0, 0};
  for (int j = 0; j < ns; ++j) {
    rhoD += wk->pv[j] * wk->col[j];
    for (int k = 0; k < 3; ++k) gD[k] += wk->pg[3 * j + k] * wk->col[j];
  }
  double Uo, gUo[3], lUo, Un, gUn[3], lUn;
  jastrow_one(s, R, i, R + 3 * i, &Uo, gUo, &lUo);
  jastrow_one(s, R, i, rp, &Un, gUn, &lUn);
  wk->rhoD = rhoD;
  wk->dU = Un - Uo;
  wk->rho = rhoD * exp(-(Un - Uo));
  for (int k = 0; k < 3; ++k) wk->Fp[k] = gD[k] / rhoD - gUn[k];
  wk->pend_iel = i;
  wk->valid = 1;
}

/* Accepting electron i's pending move: Sherman-Morrison
 * B <- B - B[:,p] (v - e_p)^T / rhoD with v^T = phi'^T B, or appending to the delayed
 * window; rows of A, dA, d2A replaced; log|det| += log|rhoD|. */
static void walker_accept(or_crowd* c, or_walker* wk, int w, int i) {
  const or_system* s = &c->s;
  int sp = spin_of(s, i), p = i - spin_off(s, sp), ns = spin_size(s, sp);
  double* R = c->R + (size_t)w * c->N * 3;
  if (s->update == 0) {
    double* v = dalloc(ns);
    double* bp = dalloc(ns);
    for (int l = 0; l < ns; ++l) {
      double acc = 0.0;
      for (int j = 0; j < ns; ++j) acc += wk->pv[j] * wk->B[sp][j * ns + l];
      v[l] = acc;
    }
    for (int j = 0; j < ns; ++j) bp[j] = wk->B[sp][j * ns + p];
    for (int j = 0; j < ns; ++j)
      for (int l = 0; l < ns; ++l)
        wk->B[sp][j * ns + l] -= bp[j] * (v[l] - (l == p ? 1.0 : 0.0)) / wk->rhoD;
    free(v); free(bp);
  } else {
    int m = wk->m[sp];
    wk->P[sp][m] = p;
    for (int j = 0; j < ns; ++j) wk->V[sp][m * ns + j] = wk->pv[j] - wk->A[sp][p * ns + j];
    wk->m[sp] = m + 1;
  }
  for (int j = 0; j < ns; ++j) {
    wk->A[sp][p * ns + j] = wk->pv[j];
    for (int k = 0; k < 3; ++k) wk->dA[sp][((size_t)p * ns + j) * 3 + k] = wk->pg[3 * j + k];
    wk->d2A[sp][p * ns + j] = wk->pl[j];
  }
  if (s->update != 0 && wk->m[sp] >= s->delay_rank) window_flush(c, wk, sp);
  wk->logdet[sp] += log(fabs(wk->rhoD));
  if (wk->rhoD < 0.0) wk->sign[sp] = -wk->sign[sp];
  for (int k = 0; k < 3; ++k) R[3 * i + k] = wk->rp[k];
}

/* The drift D(F) of the proposal r' = r + tau D(F) + sqrt(tau) chi (Alg. 1 line 5, read as
 * drift-diffusion).  drift == 1: the drift limited as in Umrigar, Nightingale and Runge
 * (J. Chem. Phys. 99, 2865 (1993)) with a = 1, D = F (-1 + sqrt(1 + 2 tau F^2)) /
 * (tau F^2), written as 2 F / (1 + sqrt(1 + 2 tau F^2)): D ~ F where tau F^2 is small and
 * tau |D| < sqrt(2 tau) however large F grows near a node.  drift == 2: D = F. */
static void drift_vector(const or_system* s, const double* F, double* D) {
  double scale = 0.0;
  if (s->drift == 1) {
    double f2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    scale = 2.0 / (1.0 + sqrt(1.0 + 2.0 * s->tau * f2));
  } else if (s->drift == 2) {
    scale = 1.0;
  }
  for (int k = 0; k < 3; ++k) D[k] = scale * F[k];
}

/* Metropolis(-Hastings) test, reading: A = rho^2 G(r<-r')/G(r'<-r) with
 * G(b<-a) = exp(-|b - a - tau D(F(a))|^2 / (2 tau)) when drifting, A = rho^2 otherwise;
 * accept iff u < A (strict); rho = 0 or non-finite rejects. */
static int metropolis(const or_system* s, const or_walker* wk, double u) {
  double rho = wk->rho;
  if (!(rho != 0.0) || !isfinite(rho)) return 0;
  if (s->dmc && wk->rhoD < 0.0) return 0;  /* fixed node: no crossing of a nodal surface */
  double A;
  if (s->drift) {
    double gb = 0.0, Dp[3];
    drift_vector(s, wk->Fp, Dp);
    for (int k = 0; k < 3; ++k) {
      double x = -wk->disp[k] - s->tau * Dp[k];
      gb += x * x;
    }
    double logGb = -gb / (2.0 * s->tau);
    A = rho * rho * exp(logGb - wk->logGf);
  } else {
    A = rho * rho;
  }
  return u < A;
}

/* One generation of one walker: every electron proposed once in order, then the delayed
 * windows flushed (Alg. 1 lines 3-10). Returns the number of accepted moves. */
static int walker_sweep(or_crowd* c, int w, uint32_t gen) {
  const or_system* s = &c->s;
  or_walker* wk = &c->wk[w];
  double* R = c->R + (size_t)w * c->N * 3;
  int nacc = 0;
  double sqt = sqrt(s->tau);
  for (int i = 0; i < c->N; ++i) {
    double chi[3], u, F[3] = {0, 0, 0}, D[3];
    if (s->drift) walker_grad(c, wk, w, i, F);
    drift_vector(s, F, D);
    or_move_draws(s->seed, (uint32_t)w, gen, (uint32_t)i, chi, &u);
    double rp[3], gf = 0.0;
    for (int k = 0; k < 3; ++k) {
      wk->disp[k] = s->tau * D[k] + sqt * chi[k];
      rp[k] = R[3 * i + k] + wk->disp[k];
      double x = wk->disp[k] - s->tau * D[k];
      gf += x * x;
      wk->F[k] = F[k];
    }
    wk->logGf = -gf / (2.0 * s->tau);
    walker_ratio_grad(c, wk, w, i, rp);
    if (metropolis(s, wk, u)) {
      walker_accept(c, wk, w, i);
      ++nacc;
    }
    wk->valid = 0;
  }
  for (int sp = 0; sp < 2; ++sp) window_flush(c, wk, sp);
  return nacc;
}

/* E_L of one walker from its maintained A, dA, d2A and inverse (after a flush). */
static double walker_local_energy(or_crowd* c, int w) {
  const or_system* s = &c->s;
  or_walker* wk = &c->wk[w];
  const double* R = c->R + (size_t)w * c->N * 3;
  double kin = 0.0;
  for (int sp = 0; sp < 2; ++sp) {
    window_flush(c, wk, sp);
    int ns = spin_size(s, sp), off = spin_off(s, sp);
    for (int l = 0; l < ns; ++l) {
      int i = off + l;
      double gD[3] = {0, 0, 0}, lD = 0.0;
      for (int j = 0; j < ns; ++j) {
        double bjl = wk->B[sp][j * ns + l];
        for (int k = 0; k < 3; ++k) gD[k] += wk->dA[sp][((size_t)l * ns + j) * 3 + k] * bjl;
        lD += wk->d2A[sp][(size_t)l * ns + j] * bjl;
      }
      double U, gU[3], lU;
      jastrow_one(s, R, i, R + 3 * i, &U, gU, &lU);
      double g2 = 0.0, gD2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        double g = gD[k] - gU[k];
        g2 += g * g;
        gD2 += gD[k] * gD[k];
      }
      kin += -0.5 * ((lD - gD2) - lU + g2);
    }
  }
  return kin + or_potential(s, R) + nlpp_energy(s, R, (const double* const*)wk->B);
}

/* ---- exported fine-grained calls ---------------------------------------------------- */
void or_crowd_eval_grad(or_crowd* c, int iel, double* grad) {
  for (int w = 0; w < c->W; ++w) walker_grad(c, &c->wk[w], w, iel, grad + 3 * w);
}

/* rnew [W][3] given, or NULL: drawn from the counter-based RNG at the crowd's generation.
 * Outputs (each may be NULL): ratio [W], grad [W][3] = grad_i log Psi(R'), log_ratio [W]
 * = log|ratio|, rnew_out [W][3] (the wrapped proposal). */
void or_crowd_propose(or_crowd* c, int iel, const double* rnew, double* ratio, double* grad,
                      double* log_ratio, double* rnew_out) {
  const or_system* s = &c->s;
  double sqt = sqrt(s->tau);
  for (int w = 0; w < c->W; ++w) {
    or_walker* wk = &c->wk[w];
    double* R = c->R + (size_t)w * c->N * 3;
    double rp[3], F[3] = {0, 0, 0}, D[3];
    if (s->drift) walker_grad(c, wk, w, iel, F);
    drift_vector(s, F, D);
    if (rnew) {
      double d[3];
      min_image(rnew + 3 * w, R + 3 * iel, s->L, d);
      for (int k = 0; k < 3; ++k) { rp[k] = rnew[3 * w + k]; wk->disp[k] = d[k]; }
    } else {
      double chi[3], u;
      or_move_draws(s->seed, (uint32_t)w, c->gen, (uint32_t)iel, chi, &u);
      for (int k = 0; k < 3; ++k) {
        wk->disp[k] = s->tau * D[k] + sqt * chi[k];
        rp[k] = R[3 * iel + k] + wk->disp[k];
      }
    }
    double gf = 0.0;
    for (int k = 0; k < 3; ++k) {
      double x = wk->disp[k] - s->tau * D[k];
      gf += x * x;
      wk->F[k] = F[k];
    }
    wk->logGf = -gf / (2.0 * s->tau);
    walker_ratio_grad(c, wk, w, iel, rp);
    if (ratio) ratio[w] = wk->rho;
    if (log_ratio) log_ratio[w] = log(fabs(wk->rhoD)) - wk->dU;
    if (grad) for (int k = 0; k < 3; ++k) grad[3 * w + k] = wk->Fp[k];
    if (rnew_out) for (int k = 0; k < 3; ++k) rnew_out[3 * w + k] = wk->rp[k];
  }
}

/* accept [W] given (nonzero = accept), or NULL: Metropolis with the slot-2 uniform at the
 * crowd's generation.  accepted_out [W] (may be NULL) receives the decisions.
 * Returns -1 if no proposal is pending for iel. */
int or_crowd_accept(or_crowd* c, int iel, const uint8_t* accept, uint8_t* accepted_out) {
  for (int w = 0; w < c->W; ++w)
    if (!c->wk[w].valid || c->wk[w].pend_iel != iel) return -1;
  for (int w = 0; w < c->W; ++w) {
    or_walker* wk = &c->wk[w];
    int acc;
    if (accept) acc = accept[w] != 0;
    else {
      double chi[3], u;
      or_move_draws(c->s.seed, (uint32_t)w, c->gen, (uint32_t)iel, chi, &u);
      acc = metropolis(&c->s, wk, u);
    }
    if (acc) walker_accept(c, wk, w, iel);
    if (accepted_out) accepted_out[w] = (uint8_t)acc;
    wk->valid = 0;
  }
  return 0;
}

void or_crowd_local_energy(or_crowd* c, double* eloc) {
  for (int w = 0; w < c->W; ++w) eloc[w] = walker_local_energy(c, w);
}

/* n_gen generations (Alg. 1 lines 1-11 without branching): each walker sweeps its
 * electrons, flushes, then (every n_recompute generations) recomputes A^-1 from scratch,
 * then evaluates E_L.  eloc [n_gen][W] and n_accept [W] (accumulated) may be NULL.
 * Walkers run in parallel over OpenMP threads (Alg. 2). */
int or_crowd_sweep(or_crowd* c, int n_gen, double* eloc, long long* n_accept) {
  int st = 0;
  for (int g = 0; g < n_gen; ++g) {
    uint32_t gen = c->gen;
    int do_rc = c->s.n_recompute > 0 && ((gen + 1) % (uint32_t)c->s.n_recompute) == 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : st)
    for (int w = 0; w < c->W; ++w) {
      int na = walker_sweep(c, w, gen);
      if (n_accept) n_accept[w] += na;
      if (do_rc) st |= walker_recompute(c, w);
      double e = walker_local_energy(c, w);
      if (eloc) eloc[(size_t)g * c->W + w] = e;
    }
    c->gen = gen + 1;
  }
  return st;
}

void or_crowd_get_positions(const or_crowd* c, double* R) {
  memcpy(R, c->R, sizeof(double) * c->W * c->N * 3);
}

void or_crowd_set_positions(or_crowd* c, const double* R) {
  memcpy(c->R, R, sizeof(double) * c->W * c->N * 3);
}

void or_crowd_get_logpsi(const or_crowd* c, double* logabs, int* sign) {
  for (int w = 0; w < c->W; ++w) {
    const double* R = c->R + (size_t)w * c->N * 3;
    const or_walker* wk = &c->wk[w];
    logabs[w] = wk->logdet[0] + wk->logdet[1] - or_jastrow_U(&c->s, R);
    sign[w] = wk->sign[0] * wk->sign[1];
  }
}

/* out [n][n] = the current A^-1 of one walker and spin (flushes its window). */
void or_crowd_get_inverse(or_crowd* c, int w, int sp, double* out) {
  window_flush(c, &c->wk[w], sp);
  int ns = spin_size(&c->s, sp);
  memcpy(out, c->wk[w].B[sp], sizeof(double) * ns * ns);
}

void or_crowd_get_A(const or_crowd* c, int w, int sp, double* out) {
  int ns = spin_size(&c->s, sp);
  memcpy(out, c->wk[w].A[sp], sizeof(double) * ns * ns);
}

uint32_t or_crowd_get_generation(const or_crowd* c) { return c->gen; }
void or_crowd_set_generation(or_crowd* c, uint32_t gen) { c->gen = gen; }

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel regions (n >= 1); no effect without OpenMP. */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}


/* ------------------------------------------------------------------------------------ */
/* DMC reweighting and branching (Alg. 1 lines 13-14; the paper gives no formulas, the     */
/* readings are): weight w = exp(-tau ((E_prev + E_new) / 2 - E_T)); multiplicity          */
/* M = floor(w + u) with u the walker's uniform from Philox counter (gen, N, 3, 0) and the */
/* walker's usual key; the new population lists walker 0 M_0 times, then walker 1 M_1     */
/* times, and so on, cut at `cap` entries.  Writes src[d] (the walker copied into slot d)  */
/* and the weights; returns the new population size.                                       */
/* ------------------------------------------------------------------------------------ */
int or_dmc_branch(const double* e_prev, const double* e_new, int W, int N, double tau,
                  double e_trial, uint64_t seed, uint32_t gen, int cap, int* src,
                  double* weight) {
  int d = 0;
  for (int w = 0; w < W; ++w) {
    const double wt = exp(-tau * (0.5 * (e_prev[w] + e_new[w]) - e_trial));
    weight[w] = wt;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)w ^ (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {gen, (uint32_t)N, 3u, 0u};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    const double u = u53(x[0], x[1]);
    const int M = (int)floor(wt + u);
    for (int j = 0; j < M && d < cap; ++j) src[d++] = w;
  }
  return d;
}
