/*
 * Plain CPU oracle for the block-sparse product C = alpha*A*B + beta*C.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path calls, links
 * or loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do. It shares no code with the CUDA path.
 *
 * What it computes (paper Sec. 2.1: C is produced by the rank-k updates
 * C_ij <- A_ik B_kj + C_ij over the inner blocks k; Algorithm 1 scales each
 * update by alpha; beta*C is the usual GEMM input term):
 *
 *   triples  T   = { (i,k,j) : a_mask[i][k] and b_mask[k][j] }
 *   C tiles  S_C = { (i,j) : some k with (i,k,j) in T }  union  c_mask
 *   for (i,j) in S_C:
 *       acc = 0 (r_i x c_j)
 *       for k ascending with (i,k,j) in T:   acc += A_ik * B_kj
 *       C_ij = alpha*acc + beta*C_ij      (beta == 0: C_ij is not read)
 *
 * Rounding, stated exactly so that other implementations can be compared bit
 * for bit: every scalar update of acc is one fused multiply-add
 * acc[ii][jj] = fma(A[ii][kk], B[kk][jj], acc[ii][jj]), taken in ascending k
 * block and, inside a block, ascending kk; the epilogue rounds alpha*acc and
 * beta*C separately and then adds them (compile with -ffp-contract=off).
 *
 * Storage (matches the generator module): each stored tile is row-major and
 * contiguous with leading dimension = its column-block size; offset tables are
 * int64 element offsets, -1 for an absent tile.
 *
 * Transposed operands (Sec. 2.1 notes that transposed multiplies such as C = A B^T
 * are handled the same way): bit 0 of `trans` says every A tile A_ik is stored as its
 * transpose (q_k x r_i, row-major), bit 1 that every B tile B_kj is stored as its
 * transpose (c_j x q_k). Masks and offset tables keep the (i,k) and (k,j) indexing
 * here; only the element addressing inside a tile changes, so the arithmetic, its
 * order and its rounding are the same as for untransposed storage.
 *
 * Split k (Sec. 3.2, Fig. 2: a rank-k update becomes a multiply task that forms the
 * product C^(k) = A_ik B_kj into a temporary and a task that adds the temporary into
 * C_ij, so updates of one C tile need not run one after the other). With pieces = n > 1
 * the k-list of tile (i,j), of length L, is cut into n' = min(n, L) consecutive pieces,
 * piece p taking the list positions [floor(p L / n'), floor((p+1) L / n')). Each piece
 * forms its partial sum P_p from zero with the same fused multiply-adds as acc above,
 * and the partials are reduced in piece order, acc = (...((P_0 + P_1) + P_2) + ...),
 * every addition rounded to FP64; the epilogue is unchanged. pieces <= 1 is the plain
 * definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR 1

/* Boolean product of the tile masks and the useful flop count
 * F = sum over T of 2 * r_i * c_j * q_k  (only nonzero triples are work). */
int oracle_structure(int M, int N, int K, const int32_t* r, const int32_t* c, const int32_t* q,
                     const uint8_t* a_mask, const uint8_t* b_mask, const uint8_t* c_mask_in,
                     uint8_t* c_mask_out, int64_t* n_triples, double* flops) {
  if (M < 0 || N < 0 || K < 0) return OR_ERR;
  int64_t nt = 0;
  double f = 0.0;
  for (int i = 0; i < M; i++) {
    for (int j = 0; j < N; j++) {
      int any = 0;
      for (int k = 0; k < K; k++) {
        if (a_mask[(int64_t)i * K + k] && b_mask[(int64_t)k * N + j]) {
          any = 1;
          nt++;
          f += 2.0 * (double)r[i] * (double)c[j] * (double)q[k];
        }
      }
      if (c_mask_in && c_mask_in[(int64_t)i * N + j]) any = 1;
      c_mask_out[(int64_t)i * N + j] = (uint8_t)any;
    }
  }
  *n_triples = nt;
  *flops = f;
  return OR_OK;
}

/* Ascending k-list of every C tile, in CSR form over the M*N tiles in row-major
 * tile order: tiles t have k's klist[ptr[t] .. ptr[t+1]). */
int oracle_klists(int M, int N, int K, const uint8_t* a_mask, const uint8_t* b_mask,
                  int64_t* ptr, int32_t* klist) {
  int64_t pos = 0;
  for (int i = 0; i < M; i++) {
    for (int j = 0; j < N; j++) {
      ptr[(int64_t)i * N + j] = pos;
      for (int k = 0; k < K; k++)
        if (a_mask[(int64_t)i * K + k] && b_mask[(int64_t)k * N + j]) klist[pos++] = k;
    }
  }
  ptr[(int64_t)M * N] = pos;
  return OR_OK;
}

/* acc (r_i x c_j) = sum of A_ik B_kj over the k-list positions [lo, hi) of tile
 * (i,j), from zero, one fma per scalar update (ascending k, then ascending kk). */
static void tile_sum(int i, int j, int K, int N, const int32_t* r, const int32_t* c, const int32_t* q,
                     const uint8_t* a_mask, const uint8_t* b_mask, const double* A, const int64_t* a_off,
                     const double* B, const int64_t* b_off, int64_t lo, int64_t hi, double* acc, int trans) {
  const int ri = r[i], cj = c[j];
  const int64_t nel = (int64_t)ri * cj;
  for (int64_t e = 0; e < nel; e++) acc[e] = 0.0;
  int64_t pos = -1; /* position of k in the tile's k-list */
  for (int k = 0; k < K; k++) {
    if (!(a_mask[(int64_t)i * K + k] && b_mask[(int64_t)k * N + j])) continue;
    pos++;
    if (pos < lo || pos >= hi) continue;
    const int qk = q[k];
    const double* At = A + a_off[(int64_t)i * K + k];
    const double* Bt = B + b_off[(int64_t)k * N + j];
    for (int ii = 0; ii < ri; ii++) {
      double* arow = acc + (int64_t)ii * cj;
      for (int kk = 0; kk < qk; kk++) {
        /* element (ii, kk) of A_ik and (kk, jj) of B_kj */
        const double a = (trans & 1) ? At[(int64_t)kk * ri + ii] : At[(int64_t)ii * qk + kk];
        for (int jj = 0; jj < cj; jj++) {
          const double b = (trans & 2) ? Bt[(int64_t)jj * qk + kk] : Bt[(int64_t)kk * cj + jj];
          arow[jj] = fma(a, b, arow[jj]);
        }
      }
    }
  }
}

/* One C tile: out (r_i x c_j, row-major) = alpha*acc + beta*cin, cin may be NULL
 * when beta == 0; acc and part are scratch of r_i x c_j (part is used when pieces > 1). */
static void one_tile(int i, int j, int K, int N, const int32_t* r, const int32_t* c, const int32_t* q,
                     const uint8_t* a_mask, const uint8_t* b_mask, double alpha, const double* A,
                     const int64_t* a_off, const double* B, const int64_t* b_off, double beta,
                     const double* cin, double* out, double* acc, double* part, int trans, int pieces) {
  const int ri = r[i], cj = c[j];
  const int64_t nel = (int64_t)ri * cj;
  int64_t L = 0;
  for (int k = 0; k < K; k++) L += (a_mask[(int64_t)i * K + k] && b_mask[(int64_t)k * N + j]) ? 1 : 0;
  const int64_t np = pieces > 1 ? (pieces < L ? pieces : L) : 1;
  if (np <= 1) {
    tile_sum(i, j, K, N, r, c, q, a_mask, b_mask, A, a_off, B, b_off, 0, L, acc, trans);
  } else {
    for (int64_t p = 0; p < np; p++) {
      const int64_t lo = p * L / np, hi = (p + 1) * L / np;
      tile_sum(i, j, K, N, r, c, q, a_mask, b_mask, A, a_off, B, b_off, lo, hi, p ? part : acc, trans);
      if (p)
        for (int64_t e = 0; e < nel; e++) acc[e] = acc[e] + part[e];
    }
  }
  for (int64_t e = 0; e < nel; e++) {
    double u = alpha * acc[e];
    if (beta != 0.0) {
      double v = beta * cin[e];
      out[e] = u + v;
    } else {
      out[e] = u;
    }
  }
}

/* The whole product over S_C (c_struct = the C tile set, M x N), in place on the C
 * arena. nthreads <= 0 uses the OpenMP default. */
int oracle_bsmm(int M, int N, int K, const int32_t* r, const int32_t* c, const int32_t* q,
                const uint8_t* a_mask, const uint8_t* b_mask, const uint8_t* c_struct,
                double alpha, const double* A, const int64_t* a_off, const double* B,
                const int64_t* b_off, double beta, double* C, const int64_t* c_off, int nthreads, int trans,
                int pieces) {
  int64_t maxel = 1;
  for (int i = 0; i < M; i++)
    for (int j = 0; j < N; j++) {
      int64_t e = (int64_t)r[i] * c[j];
      if (e > maxel) maxel = e;
    }
  const int64_t ntiles = (int64_t)M * N;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double* acc = (double*)malloc(sizeof(double) * (size_t)maxel);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)maxel);
    double* part = (double*)malloc(sizeof(double) * (size_t)maxel);
    if (!acc || !tmp || !part) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t t = 0; t < ntiles; t++) {
        if (!c_struct[t]) continue;
        const int i = (int)(t / N), j = (int)(t % N);
        const int64_t co = c_off[t];
        if (co < 0) {
#pragma omp atomic write
          err = 1;
          continue;
        }
        double* Ct = C + co;
        one_tile(i, j, K, N, r, c, q, a_mask, b_mask, alpha, A, a_off, B, b_off, beta, Ct, tmp, acc, part, trans,
                 pieces);
        memcpy(Ct, tmp, sizeof(double) * (size_t)((int64_t)r[i] * c[j]));
      }
    }
    free(acc);
    free(tmp);
    free(part);
  }
  return err ? OR_ERR : OR_OK;
}

/* A single C tile into a caller buffer (for sampled checks at full size);
 * cin is that tile's prior content (may be NULL when beta == 0). */
int oracle_bsmm_tile(int i, int j, int M, int N, int K, const int32_t* r, const int32_t* c,
                     const int32_t* q, const uint8_t* a_mask, const uint8_t* b_mask, double alpha,
                     const double* A, const int64_t* a_off, const double* B, const int64_t* b_off,
                     double beta, const double* cin, double* out, int trans, int pieces) {
  if (i < 0 || i >= M || j < 0 || j >= N) return OR_ERR;
  int64_t nel = (int64_t)r[i] * c[j];
  double* acc = (double*)malloc(sizeof(double) * (size_t)(nel > 0 ? nel : 1));
  double* part = (double*)malloc(sizeof(double) * (size_t)(nel > 0 ? nel : 1));
  int rc = OR_ERR;
  if (acc && part) {
    one_tile(i, j, K, N, r, c, q, a_mask, b_mask, alpha, A, a_off, B, b_off, beta, cin, out, acc, part, trans,
             pieces);
    rc = OR_OK;
  }
  free(acc);
  free(part);
  return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
