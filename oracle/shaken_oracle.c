/*
 * shaken_oracle.c -- plain, slow CPU oracle of the shaken dynamics.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py may load or call this file.  It
 * shares no code with the CUDA library (paper_1904_06257_gb300/csrc): its
 * Philox generator, exponential, thresholds, orientation, field sums and
 * observables are written here a second time, one site update at a time.
 *
 * Method: Apollonio, D'Autilia, Scoppola, Scoppola, Troiani, "Shaken dynamics:
 * an easy way to parallel Markov Chain Monte Carlo" (arXiv:1904.06257).
 *   - Hamiltonian H(sigma), Eq. (ham1), Sec. 2.
 *   - Doubling graph from an orientation E^o, Def. 2.1 and the construction
 *     that follows it, Sec. 2.
 *   - Local fields h^{1->2} (in-neighbours of x) and h^{2->1} (out-neighbours
 *     of x), below Eq. (ham21), Sec. 2.
 *   - Half steps P^{1->2}, P^{2->1} and their composition P^{sh}, Sec. 2
 *     (the law of P^{2->1} is read with its arguments as in Eq. (ham21):
 *     tau_x ~ exp(beta h^{2->1}_x(sigma') tau_x)).
 *   - Square lattice: h^{dl} = J(s_down + s_left) + q s + lambda,
 *     h^{ur} = J(s_up + s_right) + q s + lambda, Eqs. (hdl), (hur), Sec. 3;
 *     frozen set B (sigma_x = +1 for x in B), Sec. 3.
 *   - Pair Hamiltonian H(sigma^(1), sigma^(2)), Eq. (ham21) / Eq. (ham2).
 *
 * Readings fixed by this implementation (the paper does not give them):
 *   - lattice site x = (i, j), i = row, linear index i*L + j; "down" is row
 *     i-1, "left" is column j-1, "up" row i+1, "right" column j+1 (mod L).
 *     This is the orientation under which the worked trajectory in the proof
 *     of Thm 3.3 holds.
 *   - heat-bath decision: tau_x = +1 iff u < T, u a uniform 32-bit integer and
 *     T = floor(2^32 p), p = 1 / (1 + exp(-2 beta h)), all in IEEE fp64 with
 *     the exponential below (Cody-Waite reduction + degree-13 Taylor).
 *   - field rounding order: h = (Jc * s + q * sigma_x) + lambda_x, s the
 *     integer sum of the in/out neighbour spins (times +-1 couplings).
 *   - random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     key = (seed low word, seed high word), counter = (a, b, t, half + 2c).
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no FMA contraction, so the
 * rounding of every operation is the one written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon et al., SC'11, Sec. 3.3: multipliers, Weyl key     */
/* increments and the round permutation of the 4x32 variant).                */
/* ------------------------------------------------------------------------- */
#define ORC_PH_M0 0xD2511F53u
#define ORC_PH_M1 0xCD9E8D57u
#define ORC_PH_W0 0x9E3779B9u
#define ORC_PH_W1 0xBB67AE85u

void orc_philox(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]) {
  uint32_t k0 = key[0], k1 = key[1];
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += ORC_PH_W0;
      k1 += ORC_PH_W1;
    }
    uint64_t p0 = (uint64_t)ORC_PH_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)ORC_PH_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Exponential: Cody & Waite argument reduction x = k ln2 + r (ln2 split in  */
/* a 29-bit head and a tail), Taylor series of e^r to degree 13 by Horner    */
/* with fused multiply-add, scaled by 2^k.  |x| >= 64 is clamped: there the  */
/* threshold below is already 0 or 2^32 exactly.                              */
/* ------------------------------------------------------------------------- */
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_LN2_HI = 0x1.62e42ff000000p-1;
static const double ORC_LN2_LO = -0x1.718432a1b0e26p-35;
static const double ORC_INV_FACT[14] = {
    0x1.0000000000000p+0,  0x1.0000000000000p+0,  0x1.0000000000000p-1,
    0x1.5555555555555p-3,  0x1.5555555555555p-5,  0x1.1111111111111p-7,
    0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
    0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};

double orc_exp(double x) {
  if (x <= -64.0) return 0.0;
  if (x >= 64.0) return INFINITY;
  double k = nearbyint(x * ORC_INV_LN2);
  double r = (x - k * ORC_LN2_HI) - k * ORC_LN2_LO;
  double p = ORC_INV_FACT[13];
  for (int i = 12; i >= 0; --i) p = fma(p, r, ORC_INV_FACT[i]);
  return ldexp(p, (int)k);
}

/* Heat-bath probability of tau_x = +1 given field h: e^{beta h} / (2 cosh(beta h))
 * = 1 / (1 + e^{-2 beta h}) (Sec. 2, half-step laws; Sec. 3 Eq. (pasymm)),
 * and its 33-bit integer threshold T = floor(2^32 p) in [0, 2^32]. */
uint64_t orc_threshold(double h, double beta) {
  double y = beta * h;
  double e = orc_exp(-2.0 * y);
  double p = 1.0 / (1.0 + e);
  return (uint64_t)floor(ldexp(p, 32));
}

/* Local field with the rounding order fixed above. */
double orc_field(double Jc, int64_t s, double q, int sigma, double lambda) {
  double a = Jc * (double)s;
  double b = q * (double)sigma;
  return (a + b) + lambda;
}

/* ------------------------------------------------------------------------- */
/* Draws.  A lane word is 32 decisions that share counter words (a, b):      */
/*   plane draws (lattice encodings; graphs with draw = 1): W_j = Philox(key, */
/*     (a, b, t, half + 2*(j>>2)))[j&3], j = 0..31, u_k = sum_j bit_k(W_j)   */
/*     2^(31-j).                                                             */
/*   direct draws (graphs with draw = 0): u_k = W_k.                         */
/* ------------------------------------------------------------------------- */
static void orc_key(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
}

uint32_t orc_draw_plane(uint64_t seed, uint32_t a, uint32_t b, uint32_t t, uint32_t half, int k) {
  uint32_t key[2], ctr[4], out[4];
  orc_key(seed, key);
  uint32_t u = 0;
  for (int j = 0; j < 32; ++j) {
    ctr[0] = a;
    ctr[1] = b;
    ctr[2] = t;
    ctr[3] = half + 2u * (uint32_t)(j >> 2);
    orc_philox(key, ctr, out);
    uint32_t w = out[j & 3];
    u |= ((w >> k) & 1u) << (31 - j);
  }
  return u;
}

uint32_t orc_draw_direct(uint64_t seed, uint32_t a, uint32_t b, uint32_t t, uint32_t half, int k) {
  uint32_t key[2], ctr[4], out[4];
  orc_key(seed, key);
  ctr[0] = a;
  ctr[1] = b;
  ctr[2] = t;
  ctr[3] = half + 2u * (uint32_t)(k >> 2);
  orc_philox(key, ctr, out);
  return out[k & 3];
}

#define ORC_INIT_STEP 0xFFFFFFFFu

/* Lane-word coordinates of replica r, site x.  mode 0: single-replica words
 * (32 consecutive sites of one replica: int8 and bit-packed lattices);
 * mode 1: multispin words (one site of 32 consecutive replicas). */
static void orc_lane(int mode, int64_t x, int64_t r, uint32_t* a, uint32_t* b, int* k) {
  if (mode == 0) {
    *a = (uint32_t)(x >> 5);
    *b = (uint32_t)r;
    *k = (int)(x & 31);
  } else {
    *a = (uint32_t)x;
    *b = (uint32_t)(r >> 5);
    *k = (int)(r & 31);
  }
}

/* ------------------------------------------------------------------------- */
/* Lattice (Sec. 3).  Spins int8 [R][L][L], values +-1.                      */
/* ------------------------------------------------------------------------- */

/* Initial configuration: kind 0 random (sigma = +1 iff u < 2^31, drawn at
 * step 0xFFFFFFFF, half 0), 1 all plus, 2 all minus.  Frozen sites are +1. */
void orc_lattice_init(int8_t* s, int64_t L, int64_t R, const uint8_t* frozen, uint64_t seed,
                      int mode, int kind) {
  int64_t n = L * L;
  for (int64_t r = 0; r < R; ++r) {
    for (int64_t x = 0; x < n; ++x) {
      int8_t v;
      if (frozen && frozen[x]) {
        v = 1;
      } else if (kind == 1) {
        v = 1;
      } else if (kind == 2) {
        v = -1;
      } else {
        uint32_t a, b;
        int k;
        orc_lane(mode, x, r, &a, &b, &k);
        uint32_t u = orc_draw_plane(seed, a, b, ORC_INIT_STEP, 0, k);
        v = (u < 0x80000000u) ? 1 : -1;
      }
      s[r * n + x] = v;
    }
  }
}

/* One update of site x of replica r: returns tau_x.
 * half 0: P^{dl}, field from (down, left, self) of sigma (Eq. (hdl)).
 * half 1: P^{ur}, field from (up, right, self) of sigma' (Eq. (hur)). */
int orc_lattice_site(const int8_t* in_r, int64_t L, int64_t i, int64_t j, const uint8_t* frozen,
                     double J, double q, double lambda, double beta, uint64_t seed, uint32_t t,
                     int half, int mode, int64_t r) {
  int64_t x = i * L + j;
  if (frozen && frozen[x]) return 1;
  int64_t ya, yb;
  if (half == 0) {
    ya = ((i - 1 + L) % L) * L + j;
    yb = i * L + (j - 1 + L) % L;
  } else {
    ya = ((i + 1) % L) * L + j;
    yb = i * L + (j + 1) % L;
  }
  int64_t s = (int64_t)in_r[ya] + (int64_t)in_r[yb];
  double h = orc_field(J, s, q, in_r[x], lambda);
  uint64_t T = orc_threshold(h, beta);
  uint32_t a, b;
  int k;
  orc_lane(mode, x, r, &a, &b, &k);
  uint32_t u = orc_draw_plane(seed, a, b, t, (uint32_t)half, k);
  return ((uint64_t)u < T) ? 1 : -1;
}

void orc_lattice_half(const int8_t* in, int8_t* out, int64_t L, int64_t R, const uint8_t* frozen,
                      double J, double q, double lambda, const double* beta, uint64_t seed,
                      uint32_t t, int half, int mode) {
  int64_t n = L * L;
  for (int64_t r = 0; r < R; ++r)
    for (int64_t i = 0; i < L; ++i)
      for (int64_t j = 0; j < L; ++j)
        out[r * n + i * L + j] = (int8_t)orc_lattice_site(in + r * n, L, i, j, frozen, J, q,
                                                          lambda, beta[r], seed, t, half, mode, r);
}

/* n_steps full shaken steps P^{sh} = P^{dl} then P^{ur} (Sec. 3), starting at
 * step index t0.  s holds sigma_t on entry and sigma_{t0+n} on exit; sp
 * receives the last half-step configuration sigma'. */
void orc_lattice_run(int8_t* s, int8_t* sp, int64_t L, int64_t R, const uint8_t* frozen,
                     double J, double q, double lambda, const double* beta, uint64_t seed,
                     uint32_t t0, int64_t n_steps, int mode) {
  for (int64_t st = 0; st < n_steps; ++st) {
    uint32_t t = t0 + (uint32_t)st;
    orc_lattice_half(s, sp, L, R, frozen, J, q, lambda, beta, seed, t, 0, mode);
    orc_lattice_half(sp, s, L, R, frozen, J, q, lambda, beta, seed, t, 1, mode);
  }
}

/* Anneal: step t0+st uses beta_sched[st] for every replica. */
void orc_lattice_anneal(int8_t* s, int8_t* sp, int64_t L, int64_t R, const uint8_t* frozen,
                        double J, double q, double lambda, const double* beta_sched,
                        uint64_t seed, uint32_t t0, int64_t n_steps, int mode) {
  double* b = (double*)malloc(sizeof(double) * (size_t)R);
  for (int64_t st = 0; st < n_steps; ++st) {
    for (int64_t r = 0; r < R; ++r) b[r] = beta_sched[st];
    uint32_t t = t0 + (uint32_t)st;
    orc_lattice_half(s, sp, L, R, frozen, J, q, lambda, b, seed, t, 0, mode);
    orc_lattice_half(sp, s, L, R, frozen, J, q, lambda, b, seed, t, 1, mode);
  }
  free(b);
}

/* Observables of one lattice replica (integer sums; the energies follow):
 *   out[0] = M  = sum_x sigma_x
 *   out[1] = E  = sum_x sigma_x (sigma_down + sigma_left)   (each edge once)
 *   out[2] = P1 = sum_x sigma_x (sigma'_up + sigma'_right)
 *   out[3] = P2 = sum_x sigma_x sigma'_x
 *   out[4] = M2 = sum_x sigma'_x
 *   out[5] = number of edges {x,y} with sigma_x != sigma_y
 * H(sigma) = -J E - 2 lambda M (Eq. (HGibbs)); pair energy
 * H(sigma, sigma') = -(J P1 + q P2 + lambda (M + M2)) (Eq. (ham2)). */
void orc_lattice_sums(const int8_t* s, const int8_t* sp, int64_t L, int64_t out[6]) {
  for (int c = 0; c < 6; ++c) out[c] = 0;
  for (int64_t i = 0; i < L; ++i) {
    for (int64_t j = 0; j < L; ++j) {
      int64_t x = i * L + j;
      int64_t dn = ((i - 1 + L) % L) * L + j, lf = i * L + (j - 1 + L) % L;
      int64_t up = ((i + 1) % L) * L + j, rt = i * L + (j + 1) % L;
      out[0] += s[x];
      out[1] += (int64_t)s[x] * (s[dn] + s[lf]);
      out[2] += (int64_t)s[x] * (sp[up] + sp[rt]);
      out[3] += (int64_t)s[x] * sp[x];
      out[4] += sp[x];
      out[5] += (s[x] != s[dn]) + (s[x] != s[lf]);
    }
  }
}

/* ------------------------------------------------------------------------- */
/* General graphs (Sec. 2).                                                  */
/* ------------------------------------------------------------------------- */

/* Orientation E^o of the undirected edge list (Sec. 2, construction of the
 * doubling graph): rule 0 orients every edge from its smaller to its larger
 * endpoint, rule 2 keeps (u -> v) as given. */
void orc_orient(int64_t m, const int32_t* u, const int32_t* v, int rule, int32_t* tail,
                int32_t* head) {
  for (int64_t e = 0; e < m; ++e) {
    if (rule == 0) {
      tail[e] = u[e] < v[e] ? u[e] : v[e];
      head[e] = u[e] < v[e] ? v[e] : u[e];
    } else {
      tail[e] = u[e];
      head[e] = v[e];
    }
  }
}

/* Incidence lists of a half step on a graph (Sec. 2, doubling graph): for
 * half 0 (1->2) the list of x holds the oriented edges (y -> x), whose tails
 * are the in-neighbours feeding h^{1->2}_x; for half 1 (2->1) the edges
 * (x -> y), whose heads are the out-neighbours feeding h^{2->1}_x.  Built by
 * counting: the edges of x are list[start[x] .. start[x+1]) in edge order. */
void orc_incidence(int64_t n, int64_t m, const int32_t* tail, const int32_t* head, int half,
                   int64_t* start, int64_t* list) {
  for (int64_t x = 0; x <= n; ++x) start[x] = 0;
  for (int64_t e = 0; e < m; ++e) start[(half == 0 ? head[e] : tail[e]) + 1]++;
  for (int64_t x = 0; x < n; ++x) start[x + 1] += start[x];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  memcpy(fill, start, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t e = 0; e < m; ++e) list[fill[half == 0 ? head[e] : tail[e]]++] = e;
  free(fill);
}

/* Local field of x in the configuration sr [n] of one replica (the fields
 * below Eq. (ham21), Sec. 2):
 *   half 0: h_x = sum_{e: head(e)=x} J_e sigma_tail(e) + q sigma_x + lambda_x
 *   half 1: h_x = sum_{e: tail(e)=x} J_e sigma_head(e) + q sigma_x + lambda_x
 * integer_J != 0: J_e in {-1,+1}, the sum is an integer and h is rounded as
 * (s + q sigma) + lambda.  Otherwise the sum is accumulated in fp64 in edge
 * order.  start/list: orc_incidence of the same half. */
double orc_graph_field(const int8_t* sr, int64_t x, const int64_t* start, const int64_t* list,
                       const int32_t* tail, const int32_t* head, const double* J, int integer_J,
                       const double* lambda, double q, int half) {
  double h;
  if (integer_J) {
    int64_t s = 0;
    for (int64_t p = start[x]; p < start[x + 1]; ++p) {
      int64_t e = list[p];
      int32_t y = half == 0 ? tail[e] : head[e];
      s += (J[e] > 0 ? 1 : -1) * (int64_t)sr[y];
    }
    h = orc_field(1.0, s, q, sr[x], lambda[x]);
  } else {
    double acc = 0.0;
    for (int64_t p = start[x]; p < start[x + 1]; ++p) {
      int64_t e = list[p];
      int32_t y = half == 0 ? tail[e] : head[e];
      acc += J[e] * (double)sr[y];
    }
    h = (acc + q * (double)sr[x]) + lambda[x];
  }
  return h;
}

/* Draw of replica r at vertex x: lane word (a, b) = (x, r / 32), lane k = r % 32;
 * draw 0: direct (u = W_k), draw 1: bit planes (u_k = sum_j bit_k(W_j) 2^(31-j)). */
uint32_t orc_graph_draw(uint64_t seed, int64_t x, int64_t r, uint32_t t, int half, int draw) {
  if (draw == 1)
    return orc_draw_plane(seed, (uint32_t)x, (uint32_t)(r >> 5), t, (uint32_t)half, (int)(r & 31));
  return orc_draw_direct(seed, (uint32_t)x, (uint32_t)(r >> 5), t, (uint32_t)half, (int)(r & 31));
}

/* Draws of every replica and vertex of one half step into u[R][n]. */
void orc_graph_draws(uint32_t* u, int64_t n, int64_t R, uint64_t seed, uint32_t t, int half,
                     int draw) {
  for (int64_t r = 0; r < R; ++r)
    for (int64_t x = 0; x < n; ++x) u[r * n + x] = orc_graph_draw(seed, x, r, t, half, draw);
}

/* One update of vertex x of replica r on a graph: tau_x = +1 iff u < T(h_x, beta)
 * (heat-bath law of the half steps, Sec. 2); frozen vertices stay +1. */
int orc_graph_site(const int8_t* sr, int64_t x, const int64_t* start, const int64_t* list,
                   const int32_t* tail, const int32_t* head, const double* J, int integer_J,
                   const uint8_t* frozen, const double* lambda, double q, double beta,
                   uint64_t seed, uint32_t t, int half, int draw, int64_t r) {
  if (frozen && frozen[x]) return 1;
  double h = orc_graph_field(sr, x, start, list, tail, head, J, integer_J, lambda, q, half);
  uint64_t T = orc_threshold(h, beta);
  uint32_t u = orc_graph_draw(seed, x, r, t, half, draw);
  return ((uint64_t)u < T) ? 1 : -1;
}

/* One half step on a graph for all R replicas.  Spins int8 [R][n]; half 0
 * (1->2) reads the in-neighbours, half 1 (2->1) the out-neighbours (see
 * orc_graph_field); draw selects the lane layout of orc_graph_draw. */
void orc_graph_half(const int8_t* in, int8_t* out, int64_t n, int64_t m, const int32_t* tail,
                    const int32_t* head, const double* J, int integer_J, const uint8_t* frozen,
                    const double* lambda, double q, const double* beta, int64_t R, uint64_t seed,
                    uint32_t t, int half, int draw) {
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  orc_incidence(n, m, tail, head, half, start, list);
  for (int64_t r = 0; r < R; ++r)
    for (int64_t x = 0; x < n; ++x)
      out[r * n + x] = (int8_t)orc_graph_site(in + r * n, x, start, list, tail, head, J, integer_J,
                                              frozen, lambda, q, beta[r], seed, t, half, draw, r);
  free(start);
  free(list);
}

/* Fields h_x of every replica and vertex for one half step into h[R][n]
 * (orc_graph_field). */
void orc_graph_fields(const int8_t* in, double* h, int64_t n, int64_t m, const int32_t* tail,
                      const int32_t* head, const double* J, int integer_J, const double* lambda,
                      double q, int64_t R, int half) {
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  orc_incidence(n, m, tail, head, half, start, list);
  for (int64_t r = 0; r < R; ++r)
    for (int64_t x = 0; x < n; ++x)
      h[r * n + x] = orc_graph_field(in + r * n, x, start, list, tail, head, J, integer_J, lambda,
                                     q, half);
  free(start);
  free(list);
}

void orc_graph_init(int8_t* s, int64_t n, int64_t R, const uint8_t* frozen, uint64_t seed,
                    int kind) {
  for (int64_t r = 0; r < R; ++r) {
    for (int64_t x = 0; x < n; ++x) {
      int8_t v;
      if (frozen && frozen[x]) {
        v = 1;
      } else if (kind == 1) {
        v = 1;
      } else if (kind == 2) {
        v = -1;
      } else {
        uint32_t u = orc_draw_direct(seed, (uint32_t)x, (uint32_t)(r >> 5), ORC_INIT_STEP, 0,
                                     (int)(r & 31));
        v = (u < 0x80000000u) ? 1 : -1;
      }
      s[r * n + x] = v;
    }
  }
}

/* Full steps on a graph; beta_sched != NULL gives one beta per step (anneal)
 * and overrides beta; draw is the lane layout of orc_graph_draw. */
void orc_graph_run(int8_t* s, int8_t* sp, int64_t n, int64_t m, const int32_t* tail,
                   const int32_t* head, const double* J, int integer_J, const uint8_t* frozen,
                   const double* lambda, double q, const double* beta, const double* beta_sched,
                   int64_t R, uint64_t seed, uint32_t t0, int64_t n_steps, int draw) {
  double* b = (double*)malloc(sizeof(double) * (size_t)R);
  for (int64_t st = 0; st < n_steps; ++st) {
    for (int64_t r = 0; r < R; ++r) b[r] = beta_sched ? beta_sched[st] : beta[r];
    uint32_t t = t0 + (uint32_t)st;
    orc_graph_half(s, sp, n, m, tail, head, J, integer_J, frozen, lambda, q, b, R, seed, t, 0, draw);
    orc_graph_half(sp, s, n, m, tail, head, J, integer_J, frozen, lambda, q, b, R, seed, t, 1, draw);
  }
  free(b);
}

/* Observables of one graph replica:
 *   out[0] = sum_x sigma_x
 *   out[1] = sum_{(y->x) in E^o} J sigma_x sigma_y          (each edge once)
 *   out[2] = sum_x lambda_x sigma_x
 *   out[3] = sum_{(x->y) in E^o} J sigma_x sigma'_y
 *   out[4] = sum_x sigma_x sigma'_x
 *   out[5] = sum_x lambda_x sigma'_x
 *   out[6] = number of edges with sigma_x != sigma_y
 * H(sigma) = -out[1] - 2 out[2] (Eq. (ham1)); pair energy
 * H(sigma, sigma') = -(out[3] + q out[4] + out[2] + out[5]) (Eq. (ham21)). */
void orc_graph_sums(const int8_t* s, const int8_t* sp, int64_t n, int64_t m, const int32_t* tail,
                    const int32_t* head, const double* J, const double* lambda, double out[7]) {
  for (int c = 0; c < 7; ++c) out[c] = 0.0;
  for (int64_t x = 0; x < n; ++x) {
    out[0] += s[x];
    out[2] += lambda[x] * s[x];
    out[4] += (double)(s[x] * sp[x]);
    out[5] += lambda[x] * sp[x];
  }
  for (int64_t e = 0; e < m; ++e) {
    out[1] += J[e] * (double)(s[tail[e]] * s[head[e]]);
    out[3] += J[e] * (double)(s[tail[e]] * sp[head[e]]);
    out[6] += (s[tail[e]] != s[head[e]]) ? 1.0 : 0.0;
  }
}
