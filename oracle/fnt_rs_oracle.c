/*
 * Plain CPU oracle for FNT-based Reed-Solomon erasure codes over F_65537
 * (Soro & Lacan, "FNT-based Reed-Solomon Erasure Codes").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Every product is taken in 64-bit integers and reduced with the C `%`
 * operator: no Fermat-specific reduction tricks are used here, so that a
 * reader can check each line against the paper's definitions by eye.
 *
 * Functions and the passages they follow:
 *   orc_root         root of order n = 2^i is 3^(2^(16-i))        (Sec. II.B)
 *   orc_dft          DFT / inverse DFT by definition               (Sec. II.A, DFT displays)
 *   orc_encode       e_i = s(r^i), Horner evaluation per codeword  (Sec. II.B, e_i = s(r^i);
 *                    FNT as evaluation on 1, r, ..., r^{n-1}: Sec. II.A)
 *   orc_encode_rows  the same at selected rows only
 *   orc_pattern      A(x) = prod_j (x - x_j), A'(x), A'(x_i), and
 *                    1 / A'(x_i) = 1 / A_i(x_i)                    (Sec. II.B, Lagrange
 *                                                                   rewrite and derivative identity)
 *   orc_decode       P(x) = sum_i v_i A_i(x) / A_i(x_i) with
 *                    A_i = A / (x - x_i) by synthetic division     (Sec. II.B, Lagrange formula)
 *   orc_interpolate  the same P with all its coefficients kept as elements of F_p
 *   orc_encode_sys   systematic code: intermediate symbols = the interpolant of the source at
 *                    the first k points r^0..r^(k-1), encoded = its values at r^j
 *                    (Sec. II, "Toward a systematic code"); j < n_out (puncturing, Sec. II.B)
 *   orc_decode_sys   systematic decode: interpolate the first k received points, then the
 *                    source is the interpolant's value at r^0..r^(k-1) (same section)
 *
 * Readings where the paper is silent: the first k entries of `positions`
 * are the interpolation points (Sec. II.B, "first k evaluation points
 * received"); an interpolated coefficient equal to 65536 cannot be a 16-bit
 * source symbol, so the decoder writes 0 there and reports ORC_RANGE;
 * received values are taken modulo p.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_P 65537u

enum { ORC_OK = 0, ORC_ARG = -1, ORC_POSITIONS = -2, ORC_RANGE = -3 };

static uint32_t orc_mul(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a * (uint64_t)b) % ORC_P);
}

static uint32_t orc_add(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a + (uint64_t)b) % ORC_P);
}

static uint32_t orc_sub(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a + ORC_P - (uint64_t)(b % ORC_P)) % ORC_P);
}

uint32_t orc_pow(uint32_t a, uint64_t e) {
  uint64_t result = 1, base = a % ORC_P;
  while (e) {
    if (e & 1) result = (result * base) % ORC_P;
    base = (base * base) % ORC_P;
    e >>= 1;
  }
  return (uint32_t)result;
}

/* Fermat inverse a^(p-2); 0 has no inverse and maps to 0. */
uint32_t orc_inv(uint32_t a) { return orc_pow(a, ORC_P - 2); }

static int is_pow2_n(uint32_t n) { return n >= 1 && n <= 65536 && (n & (n - 1)) == 0; }

/* Sec. II.B: 3 has order 2^16, so r = 3^(2^(16-i)) has order n = 2^i. */
uint32_t orc_root(uint32_t n) {
  if (!is_pow2_n(n)) return 0;
  return orc_pow(3, 65536u / n);
}

/*
 * DFT by definition (Sec. II.A):
 *   forward  A_j = sum_i a_i r^(ij)
 *   inverse  a_j = n^-1 sum_i A_i r^(-ij)
 * in: [n][ld_in] u32 (column c is one vector), out: [n][ld_out] u32.
 */
int orc_dft(uint32_t n, uint32_t root, int inverse, const uint32_t* in, size_t ld_in,
            uint32_t* out, size_t ld_out, size_t W, int nthreads) {
  if (!is_pow2_n(n) || !in || !out) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  if (inverse) r = orc_inv(r);
  uint32_t ninv = orc_inv(n % ORC_P);
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long c = 0; c < (long long)W; ++c) {
    for (uint32_t j = 0; j < n; ++j) {
      uint32_t rj = orc_pow(r, j);      /* r^j */
      uint32_t rij = 1;                 /* r^(ij), i = 0 */
      uint32_t acc = 0;
      for (uint32_t i = 0; i < n; ++i) {
        acc = orc_add(acc, orc_mul(in[(size_t)i * ld_in + c] % ORC_P, rij));
        rij = orc_mul(rij, rj);
      }
      out[(size_t)j * ld_out + c] = inverse ? orc_mul(acc, ninv) : acc;
    }
  }
  return ORC_OK;
}

/*
 * Non-systematic encoding (Sec. II.B): e_i = s(r^i), 0 <= i < n, where s(x)
 * has the k source symbols as coefficients.  Horner evaluation.
 * src: [k][ld_src] u16 (row i = source symbol i of every codeword),
 * enc: [n][ld_enc] u32 in [0, 65536].
 */
int orc_encode(uint32_t n, uint32_t k, uint32_t root, const uint16_t* src, size_t ld_src,
               uint32_t* enc, size_t ld_enc, size_t W, int nthreads) {
  if (!is_pow2_n(n) || k < 1 || k > n || !src || !enc) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long c = 0; c < (long long)W; ++c) {
    uint32_t x = 1; /* r^j */
    for (uint32_t j = 0; j < n; ++j) {
      uint32_t acc = 0;
      for (uint32_t i = k; i-- > 0;) acc = orc_add(orc_mul(acc, x), src[(size_t)i * ld_src + c]);
      enc[(size_t)j * ld_enc + c] = acc;
      x = orc_mul(x, r);
    }
  }
  return ORC_OK;
}

/*
 * The same definition, e_j = s(r^j), evaluated only at the rows listed in
 * `rows` (Horner, O(k) per entry); out: [nrows][ld_out].
 */
int orc_encode_rows(uint32_t n, uint32_t k, uint32_t root, const uint16_t* src, size_t ld_src,
                    const uint32_t* rows, uint32_t nrows, uint32_t* out, size_t ld_out, size_t W,
                    int nthreads) {
  if (!is_pow2_n(n) || k < 1 || k > n || !src || !out || !rows) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long c = 0; c < (long long)W; ++c) {
    for (uint32_t t = 0; t < nrows; ++t) {
      uint32_t x = orc_pow(r, rows[t]);
      uint32_t acc = 0;
      for (uint32_t i = k; i-- > 0;) acc = orc_add(orc_mul(acc, x), src[(size_t)i * ld_src + c]);
      out[(size_t)t * ld_out + c] = acc;
    }
  }
  return ORC_OK;
}

/* Positions must be distinct, below n, and at least k of them. */
static int check_positions(uint32_t n, uint32_t k, const uint32_t* pos, uint32_t npos) {
  if (npos < k) return ORC_POSITIONS;
  unsigned char* seen = (unsigned char*)calloc(n, 1);
  if (!seen) return ORC_ARG;
  int rc = ORC_OK;
  for (uint32_t i = 0; i < npos; ++i) {
    if (pos[i] >= n || seen[pos[i]]) { rc = ORC_POSITIONS; break; }
    seen[pos[i]] = 1;
  }
  free(seen);
  return rc;
}

/*
 * Per-pattern quantities (Sec. II.B, steps 1-3 of the interpolation):
 *   x_i = r^(z_i) for the first k positions z_i,
 *   A(x) = prod_i (x - x_i)          -> A_out[0..k] (A_out[k] = 1),
 *   A'(x_i) = A_i(x_i)               -> evaluated by Horner on A',
 *   w_i = 1 / A'(x_i)                -> w_out[0..k-1].
 * A is built by multiplying in one linear factor at a time.
 */
int orc_pattern(uint32_t n, uint32_t k, uint32_t root, const uint32_t* positions, uint32_t npos,
                uint32_t* A_out, uint32_t* dA_at_x_out, uint32_t* w_out) {
  if (!is_pow2_n(n) || k < 1 || k > n || !positions) return ORC_ARG;
  int rc = check_positions(n, k, positions, npos);
  if (rc) return rc;
  uint32_t r = root ? root : orc_root(n);
  uint32_t* A = (uint32_t*)calloc((size_t)k + 1, sizeof(uint32_t));
  uint32_t* x = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
  if (!A || !x) { free(A); free(x); return ORC_ARG; }
  for (uint32_t i = 0; i < k; ++i) x[i] = orc_pow(r, positions[i]);
  /* A starts as the constant 1; multiply by (x - x_i) for each i. */
  A[0] = 1;
  for (uint32_t i = 0; i < k; ++i) {
    /* new A_j = A_{j-1} - x_i A_j, degree grows from i to i+1 */
    for (uint32_t j = i + 1; j > 0; --j) A[j] = orc_sub(A[j - 1], orc_mul(x[i], A[j]));
    A[0] = orc_sub(0, orc_mul(x[i], A[0]));
  }
  for (uint32_t i = 0; i < k; ++i) {
    /* A'(x) = sum_j j A_j x^(j-1), Horner at x_i */
    uint32_t acc = 0;
    for (uint32_t j = k; j >= 1; --j) acc = orc_add(orc_mul(acc, x[i]), orc_mul(j % ORC_P, A[j]));
    if (dA_at_x_out) dA_at_x_out[i] = acc;
    if (w_out) w_out[i] = orc_inv(acc);
  }
  if (A_out) memcpy(A_out, A, ((size_t)k + 1) * sizeof(uint32_t));
  free(A);
  free(x);
  return ORC_OK;
}

/*
 * Erasure decoding by Lagrange interpolation (Sec. II.B):
 *   P(x) = sum_i v_i A_i(x) / A_i(x_i),  A_i(x) = A(x) / (x - x_i),
 * over the first k received points; the coefficients of P are the source.
 * recv: [npos][ld_recv] u32, row i holds the symbols received at position
 * positions[i].  out: [k][ld_out] u16.  *range_flag is set to 1 when a
 * coefficient equals 65536 (written as 0).
 */
int orc_decode(uint32_t n, uint32_t k, uint32_t root, const uint32_t* recv, size_t ld_recv,
               const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out, size_t W,
               int* range_flag, int nthreads) {
  if (!is_pow2_n(n) || k < 1 || k > n || !recv || !out) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  uint32_t* A = (uint32_t*)malloc(((size_t)k + 1) * sizeof(uint32_t));
  uint32_t* w = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
  if (!A || !w) { free(A); free(w); return ORC_ARG; }
  int rc = orc_pattern(n, k, r, positions, npos, A, NULL, w);
  if (rc) { free(A); free(w); return rc; }
  int flag = 0;
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(| : flag)
#endif
  for (long long c = 0; c < (long long)W; ++c) {
    uint32_t* P = (uint32_t*)calloc(k, sizeof(uint32_t));
    uint32_t* Q = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
    for (uint32_t i = 0; i < k; ++i) {
      uint32_t xi = orc_pow(r, positions[i]);
      /* synthetic division: Q = A / (x - x_i), deg Q = k - 1 */
      Q[k - 1] = A[k];
      for (uint32_t j = k - 1; j >= 1; --j) Q[j - 1] = orc_add(A[j], orc_mul(xi, Q[j]));
      uint32_t coef = orc_mul(recv[(size_t)i * ld_recv + c] % ORC_P, w[i]);
      for (uint32_t j = 0; j < k; ++j) P[j] = orc_add(P[j], orc_mul(coef, Q[j]));
    }
    for (uint32_t j = 0; j < k; ++j) {
      if (P[j] == 65536u) { flag = 1; out[(size_t)j * ld_out + c] = 0; }
      else out[(size_t)j * ld_out + c] = (uint16_t)P[j];
    }
    free(P);
    free(Q);
  }
  free(A);
  free(w);
  if (range_flag) *range_flag = flag;
  return flag ? ORC_RANGE : ORC_OK;
}

/*
 * Lagrange interpolation as orc_decode, with the coefficients of P kept as
 * elements of F_p (u32 in [0, 65536]): coef [k][ld_coef].
 */
int orc_interpolate(uint32_t n, uint32_t k, uint32_t root, const uint32_t* recv, size_t ld_recv,
                    const uint32_t* positions, uint32_t npos, uint32_t* coef, size_t ld_coef,
                    size_t W, int nthreads) {
  if (!is_pow2_n(n) || k < 1 || k > n || !recv || !coef) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  uint32_t* A = (uint32_t*)malloc(((size_t)k + 1) * sizeof(uint32_t));
  uint32_t* w = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
  if (!A || !w) { free(A); free(w); return ORC_ARG; }
  int rc = orc_pattern(n, k, r, positions, npos, A, NULL, w);
  if (rc) { free(A); free(w); return rc; }
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long c = 0; c < (long long)W; ++c) {
    uint32_t* P = (uint32_t*)calloc(k, sizeof(uint32_t));
    uint32_t* Q = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
    for (uint32_t i = 0; i < k; ++i) {
      uint32_t xi = orc_pow(r, positions[i]);
      Q[k - 1] = A[k];
      for (uint32_t j = k - 1; j >= 1; --j) Q[j - 1] = orc_add(A[j], orc_mul(xi, Q[j]));
      uint32_t cf = orc_mul(recv[(size_t)i * ld_recv + c] % ORC_P, w[i]);
      for (uint32_t j = 0; j < k; ++j) P[j] = orc_add(P[j], orc_mul(cf, Q[j]));
    }
    for (uint32_t j = 0; j < k; ++j) coef[(size_t)j * ld_coef + c] = P[j];
    free(P);
    free(Q);
  }
  free(A);
  free(w);
  return ORC_OK;
}

/* Value at r^j (j < n_rows) of the polynomial with coefficients coef [k][ld] (Horner). */
static void eval_rows(uint32_t r, uint32_t k, const uint32_t* coef, size_t ld_coef,
                      uint32_t n_rows, uint32_t* out, size_t ld_out, size_t W, int nthreads) {
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (long long c = 0; c < (long long)W; ++c) {
    uint32_t x = 1;
    for (uint32_t j = 0; j < n_rows; ++j) {
      uint32_t acc = 0;
      for (uint32_t i = k; i-- > 0;) acc = orc_add(orc_mul(acc, x), coef[(size_t)i * ld_coef + c]);
      out[(size_t)j * ld_out + c] = acc;
      x = orc_mul(x, r);
    }
  }
}

/*
 * Systematic encode: i(x) = the interpolant of s_0..s_{k-1} at r^0..r^(k-1),
 * enc[j] = i(r^j) for j < n_out (so enc[j] = s_j for j < k).
 * src [k][ld_src] u16, enc [n_out][ld_enc] u32; k <= n_out <= n.
 */
int orc_encode_sys(uint32_t n, uint32_t k, uint32_t root, const uint16_t* src, size_t ld_src,
                   uint32_t n_out, uint32_t* enc, size_t ld_enc, size_t W, int nthreads) {
  if (!is_pow2_n(n) || k < 1 || k > n || n_out < k || n_out > n || !src || !enc) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  uint32_t* pos = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
  uint32_t* vals = (uint32_t*)malloc((size_t)k * W * sizeof(uint32_t));
  uint32_t* coef = (uint32_t*)malloc((size_t)k * W * sizeof(uint32_t));
  int rc = ORC_ARG;
  if (pos && vals && coef) {
    for (uint32_t i = 0; i < k; ++i) pos[i] = i;
    for (size_t i = 0; i < k; ++i)
      for (size_t c = 0; c < W; ++c) vals[i * W + c] = src[i * ld_src + c];
    rc = orc_interpolate(n, k, r, vals, W, pos, k, coef, W, W, nthreads);
    if (rc == ORC_OK) eval_rows(r, k, coef, W, n_out, enc, ld_enc, W, nthreads);
  }
  free(pos);
  free(vals);
  free(coef);
  return rc;
}

/*
 * Systematic decode: i(x) = the interpolant of the first k received points,
 * out[j] = i(r^j) for j < k (u16; a value 65536 is written as 0 and sets
 * *range_flag).  recv [npos][ld_recv] u32 as for orc_decode.
 */
int orc_decode_sys(uint32_t n, uint32_t k, uint32_t root, const uint32_t* recv, size_t ld_recv,
                   const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out,
                   size_t W, int* range_flag, int nthreads) {
  if (!is_pow2_n(n) || k < 1 || k > n || !recv || !out) return ORC_ARG;
  uint32_t r = root ? root : orc_root(n);
  uint32_t* coef = (uint32_t*)malloc((size_t)k * W * sizeof(uint32_t));
  uint32_t* vals = (uint32_t*)malloc((size_t)k * W * sizeof(uint32_t));
  if (!coef || !vals) { free(coef); free(vals); return ORC_ARG; }
  int rc = orc_interpolate(n, k, r, recv, ld_recv, positions, npos, coef, W, W, nthreads);
  int flag = 0;
  if (rc == ORC_OK) {
    eval_rows(r, k, coef, W, k, vals, W, W, nthreads);
    for (size_t j = 0; j < k; ++j)
      for (size_t c = 0; c < W; ++c) {
        const uint32_t v = vals[j * W + c];
        if (v == 65536u) { flag = 1; out[j * ld_out + c] = 0; }
        else out[j * ld_out + c] = (uint16_t)v;
      }
  }
  free(coef);
  free(vals);
  if (range_flag) *range_flag = flag;
  if (rc) return rc;
  return flag ? ORC_RANGE : ORC_OK;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
