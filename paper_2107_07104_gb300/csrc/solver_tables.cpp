// Host-side coefficient tables of the partitioned tridiagonal solve used by
// the split-step kernel for the Crank-Nicolson diffusion halves.
//
// System (eq:lumping_crank_nicolson_2 with lumped linear elements,
// sec:mass_lumping, Neumann ends eq:monodomain_bc1), r = c dt_1d / h^2:
//   row 0:          (1 + r) x0 - r x1                    = d0
//   row i interior: -r/2 x(i-1) + (1 + r) xi - r/2 x(i+1) = di
//   row N-1:        -r x(N-2) + (1 + r) x(N-1)           = d(N-1)
// The thesis solves it per fiber with the Thomas algorithm
// (sec:improved_parallel_solver_for_fiber_based).  On the GPU each fiber is
// split into chunks of K consecutive rows, one chunk per thread:
//   1. Thomas-style forward elimination inside the chunk expresses every row
//      j = 1..K-1 as  alpha_j x_s + x_j + gamma_j x_(j+1) = delta_j, where
//      x_s is the chunk's first unknown;
//   2. back substitution expresses the interior rows as
//      x_j = delta'_j - alpha'_j x_s - beta_j x_e  (x_e: the last unknown);
//   3. the chunk's first and last rows become a reduced tridiagonal system
//      in (x_s, x_e) of all chunks; one step of cyclic reduction removes the
//      x_s unknowns, and parallel cyclic reduction (PCR) over the chunks
//      solves for x_e;
//   4. x_s and the interior unknowns follow from steps 1-2.
// Everything except the right-hand-side terms depends on the matrix only,
// which is constant in time, so it is computed here once, in FP64.  PCR
// stops after the level at which every remaining coupling (relative to the
// unit diagonal) is below a cutoff, so each dropped term moves a solution
// value by less than the cutoff times the largest |u| of the fiber:
//   - FP32 solve: 2^-32.  Its tables are rounded to FP32 (relative error
//     up to 2^-24) and its state is stored in FP32, so the dropped terms
//     are at least 256 times smaller than rounding the solve already does.
//   - FP64 solve: 2^-40, 2^16 times below the FP32 rounding of the state
//     it writes back.
// Either way the truncated solve equals the exact one up to rounding.
#include <cmath>
#include <cstdint>
#include <vector>

#include "fibers_internal.h"

namespace fib {
namespace {

struct Row {
  double a, b, c;
};

// Row i of the CN matrix of a fiber of N nodes; rows past the end are
// decoupled identity rows (padding of the last chunk and of idle threads).
Row row_of(int64_t i, int32_t N, double r) {
  if (i >= N || N == 1) return {0.0, 1.0, 0.0};
  if (i == 0) return {0.0, 1.0 + r, -r};
  if (i == N - 1) return {-r, 1.0 + r, 0.0};
  return {-0.5 * r, 1.0 + r, -0.5 * r};
}

struct Chunk {
  std::vector<double> F1, F2, G, Ap, Bt;
  double A = 0, B = 1, C = 0, c0 = 0;  // reduced first-row equation
  double ae = 0, ge = 0;               // reduced last-row equation
};

bool chunk_coeffs(const std::vector<Row>& rw, int K, Chunk* ch) {
  ch->F1.assign(K, 0.0);
  ch->F2.assign(K, 0.0);
  ch->G.assign(K, 0.0);
  ch->Ap.assign(K, 0.0);
  ch->Bt.assign(K, 0.0);
  std::vector<double> al(K, 0.0), ga(K, 0.0);
  // forward elimination, rows 1..K-1, keeping the coupling to x_s
  double den = rw[1].b;
  if (den == 0.0) return false;
  ch->F1[1] = 1.0 / den;
  ch->F2[1] = 0.0;
  al[1] = rw[1].a / den;
  ga[1] = rw[1].c / den;
  for (int j = 2; j < K; ++j) {
    den = rw[j].b - rw[j].a * ga[j - 1];
    if (den == 0.0) return false;
    ch->F1[j] = 1.0 / den;
    ch->F2[j] = rw[j].a / den;
    al[j] = -rw[j].a * al[j - 1] / den;
    ga[j] = rw[j].c / den;
  }
  for (int j = 1; j < K; ++j) ch->G[j] = ga[j];
  // back substitution, rows K-2..1, in terms of x_s and x_e
  ch->Ap[K - 2] = al[K - 2];
  ch->Bt[K - 2] = ga[K - 2];
  for (int j = K - 3; j >= 1; --j) {
    ch->Ap[j] = al[j] - ga[j] * ch->Ap[j + 1];
    ch->Bt[j] = -ga[j] * ch->Bt[j + 1];
  }
  // first row: a0 x_(prev e) + b0 x_s + c0 x_1 = d0 with x_1 eliminated
  ch->A = rw[0].a;
  ch->B = rw[0].b - rw[0].c * ch->Ap[1];
  ch->C = -rw[0].c * ch->Bt[1];
  ch->c0 = rw[0].c;
  if (ch->B == 0.0) return false;
  // last row from the forward sweep: ae x_s + x_e + ge x_(next s) = delta
  ch->ae = al[K - 1];
  ch->ge = ga[K - 1];
  return true;
}

bool chunk_at(int64_t first_row, int32_t N, double r, int K, Chunk* ch) {
  std::vector<Row> rw(K);
  for (int j = 0; j < K; ++j) rw[j] = row_of(first_row + j, N, r);
  return chunk_coeffs(rw, K, ch);
}

// Per-class reduced system: base record fields and normalised couplings.
struct Reduced {
  std::vector<double> base;  // threads x kRecBase
  std::vector<double> A, C;  // y-system couplings (unit diagonal)
};

bool reduced_system(int32_t N, double r, int K, int Tw, Reduced* out) {
  std::vector<Chunk> ch(Tw);
  for (int p = 0; p < Tw; ++p)
    if (!chunk_at((int64_t)p * K, N, r, K, &ch[p])) return false;
  out->base.assign((size_t)Tw * kRecBase, 0.0);
  out->A.assign(Tw, 0.0);
  out->C.assign(Tw, 0.0);
  for (int p = 0; p < Tw; ++p) {
    const Chunk& c = ch[p];
    const double An = (p + 1 < Tw) ? ch[p + 1].A : 0.0;
    const double Bn = (p + 1 < Tw) ? ch[p + 1].B : 1.0;
    const double Cn = (p + 1 < Tw) ? ch[p + 1].C : 0.0;
    // eliminate x_s of this chunk and of the next one from the last row
    const double b0 = 1.0 - c.ae * c.C / c.B - c.ge * An / Bn;
    if (b0 == 0.0) return false;
    const double a0 = -c.ae * c.A / c.B;
    const double cy = -c.ge * Cn / Bn;
    double* rec = &out->base[(size_t)p * kRecBase];
    rec[0] = 1.0 / c.B;
    rec[1] = c.A / c.B;
    rec[2] = c.C / c.B;
    rec[3] = c.c0;
    rec[4] = 1.0 / b0;
    rec[5] = c.ae / (c.B * b0);
    rec[6] = c.ge / (Bn * b0);
    out->A[p] = a0 / b0;
    out->C[p] = cy / b0;
  }
  return true;
}

// One PCR level at stride s on couplings (A, C); writes (ib, ka, kc) per
// thread into lvl (3 per thread) when non-null.  Returns false on a zero pivot.
bool pcr_level(std::vector<double>& A, std::vector<double>& C, int s, double* lvl) {
  const int T = (int)A.size();
  std::vector<double> A2(T), C2(T);
  for (int p = 0; p < T; ++p) {
    const double Am = (p - s >= 0) ? A[p - s] : 0.0, Cm = (p - s >= 0) ? C[p - s] : 0.0;
    const double Ap = (p + s < T) ? A[p + s] : 0.0, Cp = (p + s < T) ? C[p + s] : 0.0;
    const double bp = 1.0 - A[p] * Cm - C[p] * Ap;
    if (bp == 0.0) return false;
    A2[p] = -A[p] * Am / bp;
    C2[p] = -C[p] * Cp / bp;
    if (lvl) {
      lvl[3 * p + 0] = 1.0 / bp;
      lvl[3 * p + 1] = A[p] / bp;
      lvl[3 * p + 2] = C[p] / bp;
    }
  }
  A.swap(A2);
  C.swap(C2);
  return true;
}

double max_coupling(const std::vector<double>& A, const std::vector<double>& C) {
  double m = 0.0;
  for (size_t p = 0; p < A.size(); ++p) m = std::fmax(m, std::fabs(A[p]) + std::fabs(C[p]));
  return m;
}

int levels_needed(Reduced red, double cutoff) {
  int L = 0;
  const int T = (int)red.A.size();
  for (int s = 1; max_coupling(red.A, red.C) > cutoff && s < T && L < kMaxLevels; s *= 2, ++L)
    if (!pcr_level(red.A, red.C, s, nullptr)) return -1;
  return L;
}

}  // namespace

bool build_solver_tables(int K, double r, const std::vector<int32_t>& lengths,
                         const std::vector<int32_t>& threads_per_class, bool fp64_solve, SolverTables* out) {
  if (K < 4 || lengths.size() != threads_per_class.size()) return false;
  out->K = K;
  const size_t nc = lengths.size();
  std::vector<Reduced> red(nc);
  int L = 0;
  for (size_t i = 0; i < nc; ++i) {
    const int32_t N = lengths[i];
    const double rf = N > 1 ? r : 0.0;
    if (!reduced_system(N, rf, K, threads_per_class[i], &red[i])) return false;
    const int l = levels_needed(red[i], fp64_solve ? 0x1p-40 : 0x1p-32);
    if (l < 0) return false;
    L = l > L ? l : L;
  }
  out->levels = L;
  out->rec_stride = kRecBase + kRecPerLevel * L;
  // row sets: interior chunk first, then one last-chunk set per class
  out->rows.assign((size_t)(1 + nc) * K * kCoefPerRow, 0.0);
  out->class_last.assign(nc, 0);
  out->class_rec.assign(nc, 0);
  auto put_set = [&](const Chunk& c, size_t at) {
    for (int j = 0; j < K; ++j) {
      double* q = &out->rows[at + (size_t)j * kCoefPerRow];
      q[0] = c.F1[j];
      q[1] = c.F2[j];
      q[2] = c.G[j];
      q[3] = c.Ap[j];
      q[4] = c.Bt[j];
    }
  };
  {
    std::vector<Row> rw(K, Row{-0.5 * r, 1.0 + r, -0.5 * r});
    Chunk c;
    if (!chunk_coeffs(rw, K, &c)) return false;
    put_set(c, 0);
  }
  size_t rec_total = 0;
  for (size_t i = 0; i < nc; ++i) rec_total += (size_t)threads_per_class[i] * out->rec_stride;
  out->recs.assign(rec_total, 0.0);
  size_t rec_at = 0;
  for (size_t i = 0; i < nc; ++i) {
    const int32_t N = lengths[i];
    const double rf = N > 1 ? r : 0.0;
    const int Tw = threads_per_class[i];
    const int Tf = (int)((N + K - 1) / K);
    Chunk last;
    if (!chunk_at((int64_t)(Tf - 1) * K, N, rf, K, &last)) return false;
    const size_t set_at = (size_t)(1 + i) * K * kCoefPerRow;
    put_set(last, set_at);
    out->class_last[i] = (int64_t)set_at;
    out->class_rec[i] = (int64_t)rec_at;
    Reduced rd = red[i];
    std::vector<double> lv((size_t)3 * Tw);
    for (int p = 0; p < Tw; ++p)
      for (int k = 0; k < kRecBase; ++k)
        out->recs[rec_at + (size_t)p * out->rec_stride + k] = rd.base[(size_t)p * kRecBase + k];
    for (int l = 0, s = 1; l < L; ++l, s *= 2) {
      if (!pcr_level(rd.A, rd.C, s, lv.data())) return false;
      for (int p = 0; p < Tw; ++p)
        for (int k = 0; k < 3; ++k)
          out->recs[rec_at + (size_t)p * out->rec_stride + kRecBase + 3 * l + k] = lv[(size_t)3 * p + k];
    }
    rec_at += (size_t)Tw * out->rec_stride;
  }
  return true;
}

}  // namespace fib
