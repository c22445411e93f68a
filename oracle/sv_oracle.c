/*
 * sv_oracle.c -- plain complex128 CPU state-vector oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg call this code; the CUDA library never does, and the two
 * share no source, header, table or helper.
 *
 * What it computes is the plain definition of exact state-vector simulation:
 *
 *   - gate matrices from their definitions (Sec. 4.2 gate table; rotations
 *     R_P(theta) = exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P,
 *     Sec. 9.1), built in double precision (Sec. 3.3, Sec. 5.2);
 *   - gate application by grouping the 2^k amplitudes that differ only on the
 *     target qubits (Sec. 5.3, the gather--multiply--scatter equation),
 *     with the group members found by inserting zero bits at the target
 *     positions; controls (with control states) filter groups (Sec. 4.2);
 *   - Pauli-string action P|b> = i^{nY} (-1)^{popcount(b & z)} |b xor x>
 *     and expectations <psi|P|psi> term by term (Sec. 4.4, Pauli equation);
 *   - the gradient of f = <psi|H|psi> by the adjoint recursion (reverse sweep
 *     over gates, g = Im <lambda|G|psi_k> for U = exp(-i theta G / 2));
 *   - the paper's gate fusion: consecutive gates joined, in order, while the
 *     union of their qubits stays within k (Sec. 4.3 `fuse`, Sec. 9.2);
 *     a block's matrix is the ordered product of its embedded gates;
 *   - measurement: p_i = x_i^2 + y_i^2 for psi_i = x_i + i y_i, normalised
 *     (Sec. 5.3, measurement equation), and finite-shot draws of basis
 *     indices from it by the inverse of its cumulative distribution, the
 *     uniform draws given by the caller (see og_sample).
 *
 * No blocking, no fusion beyond the above, no reordering.  The group loops
 * carry an OpenMP pragma (each group is disjoint), which changes nothing in
 * the arithmetic of any amplitude.
 *
 * Bit order: qubit q is bit q of the basis index.  For a k-qubit matrix,
 * targets[0] is the least significant bit of its row/column index.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Gate kinds (the families of the Sec. 4.2 gate table that this path runs). */
enum {
  OK_I = 0, OK_X, OK_Y, OK_Z, OK_H, OK_S, OK_SDG, OK_T, OK_TDG, OK_SX,
  OK_RX, OK_RY, OK_RZ, OK_P, OK_U2, OK_U3,
  OK_SWAP, OK_RXX, OK_RYY, OK_RZZ, OK_UNITARY, OK_EXC1, OK_EXC2, OK_NKINDS
};

#define OG_MAXQ 10

typedef struct {
  int32_t kind;
  int32_t nt;               /* number of targets */
  int32_t t[OG_MAXQ];       /* targets; t[0] = least significant matrix bit */
  int32_t nc;               /* number of controls */
  int32_t c[OG_MAXQ];       /* controls */
  int32_t cstate[OG_MAXQ];  /* control state (0/1) that enables the gate */
  double p[3];              /* angles, already bound */
  int32_t slot;             /* parameter slot of p[0] (gradient), or -1 */
  const double* mat;        /* OK_UNITARY: row-major (2^nt)^2 (re, im) pairs */
} og_gate;

/* ------------------------------------------------------------ matrices */

static void pauli_1q(int which, cplx m[4]) {
  /* which: 0 = I, 1 = X, 2 = Y, 3 = Z; row-major */
  static const double re[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, 0, 0, 0}, {1, 0, 0, -1}};
  static const double im[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, -1, 1, 0}, {0, 0, 0, 0}};
  for (int i = 0; i < 4; i++) m[i] = re[which][i] + I * im[which][i];
}

/* exp(-i theta P / 2) for P = P_a (x) P_b acting on (t[1], t[0]) when two
 * letters are given, or P_a alone; uses P^2 = I. */
static int rotation(int a, int b, double theta, cplx* U) {
  double c = cos(theta / 2.0), s = sin(theta / 2.0);
  if (b < 0) {
    cplx P[4];
    pauli_1q(a, P);
    for (int r = 0; r < 2; r++)
      for (int q = 0; q < 2; q++) U[r * 2 + q] = (r == q ? c : 0.0) - I * s * P[r * 2 + q];
    return 2;
  }
  cplx Pa[4], Pb[4];
  pauli_1q(a, Pa);
  pauli_1q(b, Pb);
  /* row index j = b0 + 2 b1, b0 the bit of t[0] (letter b), b1 of t[1] (letter a) */
  for (int r = 0; r < 4; r++)
    for (int q = 0; q < 4; q++) {
      cplx pp = Pa[(r >> 1) * 2 + (q >> 1)] * Pb[(r & 1) * 2 + (q & 1)];
      U[r * 4 + q] = (r == q ? c : 0.0) - I * s * pp;
    }
  return 4;
}

/* Writes the (2^nt x 2^nt) matrix of the gate, without its controls.
 * Returns the dimension, or 0 for an unknown kind. */
int og_gate_matrix(const og_gate* g, double* out_re_im) {
  cplx U[1024];
  int d = 0;
  const double r2 = 1.0 / sqrt(2.0);
  switch (g->kind) {
    case OK_I: pauli_1q(0, U); d = 2; break;
    case OK_X: pauli_1q(1, U); d = 2; break;
    case OK_Y: pauli_1q(2, U); d = 2; break;
    case OK_Z: pauli_1q(3, U); d = 2; break;
    case OK_H: U[0] = r2; U[1] = r2; U[2] = r2; U[3] = -r2; d = 2; break;
    case OK_S: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = I; d = 2; break;
    case OK_SDG: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = -I; d = 2; break;
    case OK_T: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(I * M_PI / 4.0); d = 2; break;
    case OK_TDG: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(-I * M_PI / 4.0); d = 2; break;
    case OK_SX: /* square root of X */
      U[0] = 0.5 * (1 + I); U[1] = 0.5 * (1 - I); U[2] = 0.5 * (1 - I); U[3] = 0.5 * (1 + I);
      d = 2; break;
    case OK_RX: d = rotation(1, -1, g->p[0], U); break;
    case OK_RY: d = rotation(2, -1, g->p[0], U); break;
    case OK_RZ: d = rotation(3, -1, g->p[0], U); break;
    case OK_P: U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(I * g->p[0]); d = 2; break;
    case OK_U2:
    case OK_U3: {
      /* OpenQASM 2: U3(th, ph, la) = [[c, -e^{i la} s], [e^{i ph} s, e^{i(ph+la)} c]],
       * U2(ph, la) = U3(pi/2, ph, la). */
      double th = g->kind == OK_U2 ? M_PI / 2.0 : g->p[0];
      double ph = g->kind == OK_U2 ? g->p[0] : g->p[1];
      double la = g->kind == OK_U2 ? g->p[1] : g->p[2];
      double c = cos(th / 2.0), s = sin(th / 2.0);
      U[0] = c;
      U[1] = -cexp(I * la) * s;
      U[2] = cexp(I * ph) * s;
      U[3] = cexp(I * (ph + la)) * c;
      d = 2;
      break;
    }
    case OK_SWAP:
      for (int i = 0; i < 16; i++) U[i] = 0;
      U[0 * 4 + 0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[3 * 4 + 3] = 1;
      d = 4; break;
    case OK_RXX: d = rotation(1, 1, g->p[0], U); break;
    case OK_RYY: d = rotation(2, 2, g->p[0], U); break;
    case OK_RZZ: d = rotation(3, 3, g->p[0], U); break;
    case OK_UNITARY:
      d = 1 << g->nt;
      for (int i = 0; i < d * d; i++) U[i] = g->mat[2 * i] + I * g->mat[2 * i + 1];
      break;
    case OK_EXC1:
    case OK_EXC2: {
      /* Single / double excitation (Sec. 4.2 gate table): the two basis states
       * that exchange the excitation(s) -- matrix indices 1, 2 (|t0 t1> =
       * |10>, |01>) or 3, 12 (t0 t1 set, t2 t3 set) -- rotate by
       * [[cos, -sin], [sin, cos]] of theta/2; every other state is unchanged. */
      d = g->kind == OK_EXC1 ? 4 : 16;
      const int a = g->kind == OK_EXC1 ? 1 : 3, b = g->kind == OK_EXC1 ? 2 : 12;
      const double c = cos(g->p[0] / 2.0), s = sin(g->p[0] / 2.0);
      for (int i = 0; i < d * d; i++) U[i] = 0;
      for (int i = 0; i < d; i++) U[i * d + i] = 1;
      U[a * d + a] = c; U[a * d + b] = -s; U[b * d + a] = s; U[b * d + b] = c;
      break;
    }
    default: return 0;
  }
  for (int i = 0; i < d * d; i++) {
    out_re_im[2 * i] = creal(U[i]);
    out_re_im[2 * i + 1] = cimag(U[i]);
  }
  return d;
}

/* ------------------------------------------------------------ application */

/* Insert a zero bit at position q of x (bits >= q move up by one). */
static uint64_t insert_zero(uint64_t x, int q) {
  uint64_t lo = x & ((1ull << q) - 1ull);
  return ((x >> q) << (q + 1)) | lo;
}

/* Applies the k-qubit matrix M (row-major, k = nt) to psi on qubits t[], on
 * the groups whose control qubits c[] hold cstate[].  One group per setting
 * of the other n-k bits (Sec. 5.3). */
void og_apply_matrix(cplx* psi, int n, int nt, const int32_t* t, int nc, const int32_t* c,
                     const int32_t* cstate, const double* M_re_im) {
  int d = 1 << nt;
  cplx M[1024];
  for (int i = 0; i < d * d; i++) M[i] = M_re_im[2 * i] + I * M_re_im[2 * i + 1];
  int sorted[OG_MAXQ];
  for (int i = 0; i < nt; i++) sorted[i] = t[i];
  for (int i = 1; i < nt; i++)
    for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; j--) {
      int tmp = sorted[j]; sorted[j] = sorted[j - 1]; sorted[j - 1] = tmp;
    }
  int64_t ngroups = (int64_t)1 << (n - nt);
#pragma omp parallel for schedule(static)
  for (int64_t grp = 0; grp < ngroups; grp++) {
    uint64_t base = (uint64_t)grp;
    for (int i = 0; i < nt; i++) base = insert_zero(base, sorted[i]);
    int on = 1;
    for (int i = 0; i < nc; i++)
      if ((int)((base >> c[i]) & 1ull) != cstate[i]) on = 0;
    if (!on) continue;
    uint64_t idx[32];
    cplx v[32];
    for (int j = 0; j < d; j++) {
      uint64_t b = base;
      for (int i = 0; i < nt; i++)
        if ((j >> i) & 1) b |= 1ull << t[i];
      idx[j] = b;
      v[j] = psi[b];
    }
    for (int r = 0; r < d; r++) {
      cplx w = 0;
      for (int q = 0; q < d; q++) w += M[r * d + q] * v[q];
      psi[idx[r]] = w;
    }
  }
}

int og_apply_gate(cplx* psi, int n, const og_gate* g) {
  double M[2 * 1024];
  if (!og_gate_matrix(g, M)) return -1;
  og_apply_matrix(psi, n, g->nt, g->t, g->nc, g->c, g->cstate, M);
  return 0;
}

void og_zero_state(cplx* psi, int n) {
  int64_t N = (int64_t)1 << n;
  for (int64_t b = 0; b < N; b++) psi[b] = 0;
  psi[0] = 1;
}

/* psi <- U_ng ... U_1 psi (psi is used as given: callers pass |0..0> or any
 * initial state). */
int og_apply_circuit(cplx* psi, int n, const og_gate* gates, int ng) {
  for (int k = 0; k < ng; k++)
    if (og_apply_gate(psi, n, &gates[k])) return -1 - k;
  return 0;
}

/* ------------------------------------------------------------ Pauli path */

static cplx i_pow(int k) {
  switch (k & 3) {
    case 0: return 1;
    case 1: return I;
    case 2: return -1;
    default: return -I;
  }
}

/* out += coeff * P psi, with P|b> = i^{nY} (-1)^{popc(b & z)} |b ^ x>
 * (Sec. 4.4).  nY = popc(x & z). */
void og_pauli_apply_add(const cplx* psi, int n, uint64_t x, uint64_t z, double coeff, cplx* out) {
  int64_t N = (int64_t)1 << n;
  cplx ph = i_pow(__builtin_popcountll(x & z)) * coeff;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < N; b++) {
    /* (P psi)[b ^ x] = phase(b) psi[b]; written as out[b] = phase(b ^ x) psi[b ^ x] */
    uint64_t src = (uint64_t)b ^ x;
    double sg = (__builtin_popcountll(src & z) & 1) ? -1.0 : 1.0;
    out[b] += ph * sg * psi[src];
  }
}

/* <psi|P|psi> = sum_b conj(psi[b ^ x]) i^{nY} (-1)^{popc(b & z)} psi[b] */
double og_expect_pauli(const cplx* psi, int n, uint64_t x, uint64_t z) {
  int64_t N = (int64_t)1 << n;
  double sre = 0.0, sim = 0.0;
#pragma omp parallel for reduction(+ : sre, sim) schedule(static)
  for (int64_t b = 0; b < N; b++) {
    double sg = (__builtin_popcountll((uint64_t)b & z) & 1) ? -1.0 : 1.0;
    cplx v = conj(psi[(uint64_t)b ^ x]) * sg * psi[b];
    sre += creal(v);
    sim += cimag(v);
  }
  cplx tot = i_pow(__builtin_popcountll(x & z)) * (sre + I * sim);
  return creal(tot);
}

/* Weighted sum of terms; also returns each term's <P_j> in per_term (may be NULL). */
double og_expect_terms(const cplx* psi, int n, const uint64_t* xs, const uint64_t* zs,
                       const double* cs, int nterms, double* per_term) {
  double tot = 0.0;
  for (int j = 0; j < nterms; j++) {
    double e = og_expect_pauli(psi, n, xs[j], zs[j]);
    if (per_term) per_term[j] = e;
    tot += cs[j] * e;
  }
  return tot;
}

/* <Z_i> for every qubit and their sum: <Z_i> = sum_b |psi_b|^2 (-1)^{b_i}. */
void og_expect_z_all(const cplx* psi, int n, double* per_qubit, double* sum) {
  double s = 0.0;
  for (int i = 0; i < n; i++) {
    per_qubit[i] = og_expect_pauli(psi, n, 0ull, 1ull << i);
    s += per_qubit[i];
  }
  *sum = s;
}

/* <a|b> = sum conj(a) b */
void og_inner(const cplx* a, const cplx* b, int n, double* re, double* im) {
  int64_t N = (int64_t)1 << n;
  double sre = 0.0, sim = 0.0;
#pragma omp parallel for reduction(+ : sre, sim) schedule(static)
  for (int64_t i = 0; i < N; i++) {
    cplx v = conj(a[i]) * b[i];
    sre += creal(v);
    sim += cimag(v);
  }
  *re = sre;
  *im = sim;
}

/* ------------------------------------------------------------ adjoint */

/* Generator G of a rotation gate written as U = exp(-i theta G / 2), acting
 * on its targets (without the control projector).  Returns its dimension,
 * or 0 for a gate that has no such generator. */
static int generator(const og_gate* g, double* G) {
  cplx P[256], Q[4], R[4];
  int d;
  switch (g->kind) {
    case OK_RX: pauli_1q(1, P); d = 2; break;
    case OK_RY: pauli_1q(2, P); d = 2; break;
    case OK_RZ: pauli_1q(3, P); d = 2; break;
    case OK_P: /* diag(1, e^{i la}) = exp(-i la (Z - I) / 2) */
      P[0] = 0; P[1] = 0; P[2] = 0; P[3] = -2; d = 2; break;
    case OK_RXX: case OK_RYY: case OK_RZZ: {
      int w = g->kind == OK_RXX ? 1 : (g->kind == OK_RYY ? 2 : 3);
      pauli_1q(w, Q);
      pauli_1q(w, R);
      for (int r = 0; r < 4; r++)
        for (int q = 0; q < 4; q++) P[r * 4 + q] = Q[(r >> 1) * 2 + (q >> 1)] * R[(r & 1) * 2 + (q & 1)];
      d = 4;
      break;
    }
    case OK_EXC1: case OK_EXC2: { /* Y on the pair of states the gate rotates */
      d = g->kind == OK_EXC1 ? 4 : 16;
      const int a = g->kind == OK_EXC1 ? 1 : 3, b = g->kind == OK_EXC1 ? 2 : 12;
      for (int i = 0; i < d * d; i++) P[i] = 0;
      P[a * d + b] = -I;
      P[b * d + a] = I;
      break;
    }
    default: return 0;
  }
  for (int i = 0; i < d * d; i++) { G[2 * i] = creal(P[i]); G[2 * i + 1] = cimag(P[i]); }
  return d;
}

static void dagger(const double* M, int d, double* Md) {
  for (int r = 0; r < d; r++)
    for (int q = 0; q < d; q++) {
      Md[2 * (r * d + q)] = M[2 * (q * d + r)];
      Md[2 * (r * d + q) + 1] = -M[2 * (q * d + r) + 1];
    }
}

/*
 * Gradient of f(theta) = <0|U^dag H U|0> (Sec. 4.2) by the adjoint recursion.
 * Forward: psi = U_N..U_1|0>.  lambda = H psi.  Then for k = N..1:
 *   if gate k is a rotation on slot s:  grad[s] += Im <lambda|G_k|psi>
 *     (psi is the state after gate k, G_k includes the control projector;
 *     this equals 2 Re <lambda|dU_k/dtheta|psi_{k-1}>)
 *   psi <- U_k^dag psi,  lambda <- U_k^dag lambda.
 * Gates with slot < 0 are constants.  Returns 0, or -1 when a gate bound to a
 * slot has no generator of the form exp(-i theta G / 2).
 */
int og_adjoint_grad(int n, const og_gate* gates, int ng, const uint64_t* xs, const uint64_t* zs,
                    const double* cs, int nterms, double* grad, int nslots, double* value) {
  int64_t N = (int64_t)1 << n;
  cplx* psi = (cplx*)malloc(sizeof(cplx) * N);
  cplx* lam = (cplx*)calloc(N, sizeof(cplx));
  cplx* proj = (cplx*)malloc(sizeof(cplx) * N);
  if (!psi || !lam || !proj) { free(psi); free(lam); free(proj); return -2; }
  for (int s = 0; s < nslots; s++) grad[s] = 0.0;
  og_zero_state(psi, n);
  if (og_apply_circuit(psi, n, gates, ng)) { free(psi); free(lam); free(proj); return -1; }
  for (int j = 0; j < nterms; j++) og_pauli_apply_add(psi, n, xs[j], zs[j], cs[j], lam);
  double vr, vi;
  og_inner(psi, lam, n, &vr, &vi);
  *value = vr;
  int rc = 0;
  for (int k = ng - 1; k >= 0; k--) {
    const og_gate* g = &gates[k];
    if (g->slot >= 0) {
      double G[2 * 256];
      if (!generator(g, G)) { rc = -1; break; }
      /* proj = (control projector (x) G) psi: zero the amplitudes that fail
       * the controls, then apply G on the targets. */
      for (int64_t b = 0; b < N; b++) {
        int on = 1;
        for (int i = 0; i < g->nc; i++)
          if ((int)(((uint64_t)b >> g->c[i]) & 1ull) != g->cstate[i]) on = 0;
        proj[b] = on ? psi[b] : 0;
      }
      og_apply_matrix(proj, n, g->nt, g->t, 0, NULL, NULL, G);
      double re, im;
      og_inner(lam, proj, n, &re, &im);
      if (g->slot < nslots) grad[g->slot] += im;
    }
    double M[2 * 1024], Md[2 * 1024];
    int d = og_gate_matrix(g, M);
    dagger(M, d, Md);
    og_apply_matrix(psi, n, g->nt, g->t, g->nc, g->c, g->cstate, Md);
    og_apply_matrix(lam, n, g->nt, g->t, g->nc, g->c, g->cstate, Md);
  }
  free(psi);
  free(lam);
  free(proj);
  return rc;
}

/* ------------------------------------------------------------ fusion */

/*
 * The paper's fusion (Sec. 4.3 `fuse`, Sec. 9.2): walk the gates in order and
 * join each into the current block while the union of the block's qubits
 * (targets and controls) stays within kmax; otherwise close the block and open
 * a new one.  No gate is moved past another.  A gate wider than kmax forms a
 * block of its own.
 *
 * Outputs, per block b: block_start[b] (first gate index; the block covers
 * gates up to block_start[b+1]-1), its sorted qubits, and its matrix: the
 * ordered product of the blocks' gates embedded in the block's 2^k space
 * (column j = the block applied to basis state j).  Returns the number of
 * blocks, or -1 if a buffer is too small.
 *
 * qubits_out: nblocks_max x OG_MAXQ ints; nq_out: nblocks_max ints;
 * mats_out: nblocks_max x (2 * 4^kcap) doubles with kcap = max(kmax, widest gate).
 */
int og_fuse(int n, const og_gate* gates, int ng, int kmax, int nblocks_max, int* block_start,
            int* nq_out, int* qubits_out, double* mats_out, int kcap) {
  (void)n;
  int nb = 0;
  int k = 0;
  while (k < ng) {
    if (nb >= nblocks_max) return -1;
    uint64_t qs = 0;
    int start = k;
    /* grow the block */
    while (k < ng) {
      uint64_t gq = 0;
      for (int i = 0; i < gates[k].nt; i++) gq |= 1ull << gates[k].t[i];
      for (int i = 0; i < gates[k].nc; i++) gq |= 1ull << gates[k].c[i];
      uint64_t u = qs | gq;
      if (k == start || __builtin_popcountll(u) <= kmax) {
        qs = u;
        k++;
        if (__builtin_popcountll(qs) > kmax) break; /* a wide gate stands alone */
      } else {
        break;
      }
    }
    int nq = __builtin_popcountll(qs);
    if (nq > kcap) return -1;
    int q[64], m = 0;
    for (int b = 0; b < 64; b++)
      if ((qs >> b) & 1ull) q[m++] = b;
    block_start[nb] = start;
    nq_out[nb] = nq;
    for (int i = 0; i < nq; i++) qubits_out[nb * OG_MAXQ + i] = q[i];
    /* block matrix, column by column: apply each gate (remapped to block-local
     * qubit indices) to the basis vector |j> of the block's nq-qubit space */
    int d = 1 << nq;
    int dcap = 1 << kcap;
    double* out = mats_out + (size_t)nb * 2 * dcap * dcap;
    cplx* col = (cplx*)malloc(sizeof(cplx) * d);
    for (int j = 0; j < d; j++) {
      for (int r = 0; r < d; r++) col[r] = (r == j) ? 1 : 0;
      for (int gi = start; gi < k; gi++) {
        og_gate lg = gates[gi];
        for (int i = 0; i < lg.nt; i++)
          for (int s = 0; s < nq; s++)
            if (q[s] == gates[gi].t[i]) lg.t[i] = s;
        for (int i = 0; i < lg.nc; i++)
          for (int s = 0; s < nq; s++)
            if (q[s] == gates[gi].c[i]) lg.c[i] = s;
        og_apply_gate(col, nq, &lg);
      }
      for (int r = 0; r < d; r++) {
        out[2 * (r * d + j)] = creal(col[r]);
        out[2 * (r * d + j) + 1] = cimag(col[r]);
      }
    }
    free(col);
    nb++;
  }
  block_start[nb] = ng;
  return nb;
}

/* ------------------------------------------------------------ measurement */

/* p_i = x_i^2 + y_i^2, divided by their sum when normalise != 0 (Sec. 5.3,
 * measurement equation).  Each p_i is rounded once per product and once for
 * the sum (this file is compiled without contraction into fused
 * multiply-adds). */
void og_probabilities(const cplx* psi, int n, int normalise, double* p) {
  const uint64_t N = 1ull << n;
  double tot = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    const double x = creal(psi[i]), y = cimag(psi[i]);
    p[i] = x * x + y * y;
    tot += p[i];
  }
  if (normalise && tot > 0.0)
    for (uint64_t i = 0; i < N; i++) p[i] /= tot;
}

/* Finite-shot draws (Sec. 5.3: basis indices drawn from the probability
 * vector).  The distribution is taken in exact integer arithmetic so that the
 * draw does not depend on the order of any floating-point sum:
 *   q_i = floor(p_i 2^61)      (p_i as in og_probabilities, not normalised),
 *   Q   = sum_i q_i,
 *   t_k = floor(floor(u_k 2^53) Q / 2^53)  for the caller's u_k in [0, 1),
 *   index_k = the smallest i with q_0 + ... + q_i > t_k.
 * Dividing every q_i by Q is the normalisation; the exact prefix sums are the
 * cumulative distribution.  Returns -1 if every q_i is 0. */
int og_sample(const cplx* psi, int n, const double* u, int64_t nshots, uint64_t* out) {
  const uint64_t N = 1ull << n;
  uint64_t* cum = (uint64_t*)malloc(sizeof(uint64_t) * N);
  if (!cum) return -2;
  uint64_t run = 0;
  for (uint64_t i = 0; i < N; i++) {
    const double x = creal(psi[i]), y = cimag(psi[i]);
    const double pi = x * x + y * y;
    run += (uint64_t)ldexp(pi, 61);
    cum[i] = run;
  }
  const uint64_t Q = run;
  if (Q == 0) {
    free(cum);
    return -1;
  }
  for (int64_t k = 0; k < nshots; k++) {
    const uint64_t m = (uint64_t)ldexp(u[k], 53);
    const uint64_t t = (uint64_t)(((unsigned __int128)m * Q) >> 53);
    uint64_t lo = 0, hi = N - 1;  /* first i with cum[i] > t */
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (cum[mid] > t)
        hi = mid;
      else
        lo = mid + 1;
    }
    out[k] = lo;
  }
  free(cum);
  return 0;
}

int og_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
