// Coupling of the fibers to a 3D mesh of the muscle: the prolongation of
// the transmembrane voltage onto a structured hexahedral mesh
// (eq:discretized_fibers_2, with the data mapping of
// sec:data_mapping_between_meshes, eq:mapping_source_target) and the static
// first bidomain equation for the extracellular potential
// (eq:discretized_fibers_3, eq:static_bidomain_rhs):
//
//     K_(sigma_i + sigma_e) phi_e = -K_(sigma_i) V3D,
//
// with linear (trilinear) finite elements, homogeneous Neumann boundaries,
// sigma_i = sigma_i_f a (x) a along the fiber axis a = z and sigma_e
// isotropic (eq:multidomain_isotropic_e).  The Neumann problem fixes phi_e up
// to a constant; the result has zero mean over the 3D nodes.
//
// GB300 layout of the work:
//   * the prolongation is a CSR matrix (3D node rows, fiber-node columns in
//     ragged order) built once on the host; one warp per row reads the
//     row's columns and factors coalesced (a row's columns are runs of
//     consecutive nodes along fibers) and reduces in FP64;
//   * the stiffness matrices are never stored: on a uniform grid with a
//     diagonal tensor the Q1 stiffness is the tensor product
//     sx Kx(x)My(x)Mz + sy Mx(x)Ky(x)Mz + sz Mx(x)My(x)Kz of 1D stiffness and
//     consistent mass rows, so each node's 27-point row is formed from six
//     3-entry 1D rows in registers;
//   * the solve is Jacobi-preconditioned conjugate gradients in FP64 in one
//     cooperative kernel: grid-wide syncs separate the matrix product, the
//     vector updates and the direction update; dot products are reduced per
//     block and summed by every block in the same order (deterministic).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fibers.h"
#include "fibers_internal.h"

namespace cg = cooperative_groups;

struct fib_emg {
  fib_ctx* fibers = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
  fib_mesh3d mesh{};
  int64_t n3 = 0;      // 3D nodes
  int64_t n_pts = 0;   // fiber nodes (ragged order)
  int64_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  float* d_w = nullptr;
  float* d_vm = nullptr;      // V of the fiber nodes, ragged order
  double* d_v3 = nullptr;     // V3D
  double* d_b = nullptr;      // right-hand side, then unused
  double* d_x = nullptr;      // phi_e
  double* d_r = nullptr;
  double* d_p = nullptr;
  double* d_q = nullptr;
  double* d_dinv = nullptr;   // inverse diagonal of K_(sigma_i + sigma_e)
  double* d_red = nullptr;    // per-block partial sums
  int* d_iters = nullptr;
  double* d_res = nullptr;    // final relative residual
  int grid = 0;               // cooperative grid size
  std::string err;
};

namespace {

constexpr int kEmgThreads = 256;

struct Stencil {  // 1D rows of stiffness (per unit conductivity) and consistent mass
  int nx, ny, nz;
  double hx, hy, hz;
  double sx, sy, sz;  // diagonal conduction tensor
};

// Entries (a = -1, 0, +1) of the assembled 1D stiffness (K) and consistent
// mass (M) rows of node i of n (uniform width h); missing neighbours are 0.
__device__ __forceinline__ void rows_1d(int i, int n, double h, double (&K)[3], double (&M)[3]) {
  const bool lo = i > 0, hi = i < n - 1;
  K[0] = lo ? -1.0 / h : 0.0;
  K[2] = hi ? -1.0 / h : 0.0;
  K[1] = ((lo ? 1.0 : 0.0) + (hi ? 1.0 : 0.0)) / h;
  M[0] = lo ? h / 6.0 : 0.0;
  M[2] = hi ? h / 6.0 : 0.0;
  M[1] = ((lo ? 2.0 : 0.0) + (hi ? 2.0 : 0.0)) * h / 6.0;
}

// y_t = (K_sigma x)_t for node t = (i, j, k).
__device__ __forceinline__ double apply_row(const Stencil& s, const double* __restrict__ x, int64_t t) {
  const int64_t nxy = (int64_t)s.nx * s.ny;
  const int k = (int)(t / nxy);
  const int64_t rem = t - (int64_t)k * nxy;
  const int j = (int)(rem / s.nx);
  const int i = (int)(rem - (int64_t)j * s.nx);
  double Kx[3], Mx[3], Ky[3], My[3], Kz[3], Mz[3];
  rows_1d(i, s.nx, s.hx, Kx, Mx);
  rows_1d(j, s.ny, s.hy, Ky, My);
  rows_1d(k, s.nz, s.hz, Kz, Mz);
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if ((c == 0 && k == 0) || (c == 2 && k == s.nz - 1)) continue;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if ((b == 0 && j == 0) || (b == 2 && j == s.ny - 1)) continue;
      const double wyz_x = My[b] * Mz[c];                 // x-stiffness term
      const double wyz_y = Ky[b] * Mz[c];                 // y-stiffness term
      const double wyz_z = My[b] * Kz[c];                 // z-stiffness term
      const int64_t base = t + (int64_t)(c - 1) * nxy + (int64_t)(b - 1) * s.nx;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if ((a == 0 && i == 0) || (a == 2 && i == s.nx - 1)) continue;
        const double w = s.sx * Kx[a] * wyz_x + s.sy * Mx[a] * wyz_y + s.sz * Mx[a] * wyz_z;
        acc = fma(w, x[base + (a - 1)], acc);
      }
    }
  }
  return acc;
}

__global__ void gather_ragged_kernel(const fib::FiberDesc* fibers, int32_t n_fibers, const float* u, float* dst,
                                     float add) {
  for (int32_t f = blockIdx.x; f < n_fibers; f += gridDim.x) {
    const fib::FiberDesc fd = fibers[f];
    for (int i = threadIdx.x; i < fd.n; i += blockDim.x) dst[fd.coff + i] = u[fd.slot + i] + add;
  }
}

// V3D_t = sum_s w_ts V_s: one warp per 3D node row.
__global__ void prolongate_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const float* __restrict__ w, const float* __restrict__ v, int64_t n3,
                                  double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n3; r += warps) {
    double acc = 0.0;
    for (int64_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) acc = fma((double)w[e], (double)v[col[e]], acc);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane == 0) out[r] = acc;
  }
}

// b = -K_(sigma_i) V3D
__global__ void rhs_kernel(Stencil si, const double* __restrict__ v3, int64_t n3, double* __restrict__ b) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = -apply_row(si, v3, t);
}

// Inverse diagonal of K_sigma.
__global__ void diag_kernel(Stencil s, int64_t n3, double* __restrict__ dinv) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nxy = (int64_t)s.nx * s.ny;
    const int k = (int)(t / nxy);
    const int64_t rem = t - (int64_t)k * nxy;
    const int j = (int)(rem / s.nx);
    const int i = (int)(rem - (int64_t)j * s.nx);
    double Kx[3], Mx[3], Ky[3], My[3], Kz[3], Mz[3];
    rows_1d(i, s.nx, s.hx, Kx, Mx);
    rows_1d(j, s.ny, s.hy, Ky, My);
    rows_1d(k, s.nz, s.hz, Kz, Mz);
    const double d = s.sx * Kx[1] * My[1] * Mz[1] + s.sy * Mx[1] * Ky[1] * Mz[1] + s.sz * Mx[1] * My[1] * Kz[1];
    dinv[t] = d > 0.0 ? 1.0 / d : 0.0;
  }
}

// Block sum of v into red[slot * gridDim.x + blockIdx.x] (thread 0 writes).
__device__ __forceinline__ void block_partial(double v, double* red, int slot, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    red[(int64_t)slot * gridDim.x + blockIdx.x] = s;
  }
  __syncthreads();
}

// Sum of all blocks' partials of a slot, in block order (every block gets
// the same bits).
__device__ __forceinline__ double grid_total(const double* red, int slot, double* sh) {
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += red[(int64_t)slot * gridDim.x + b];
  // fixed-order tree over the threads' strided sums
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

struct CgArgs {
  Stencil A;  // K_(sigma_i + sigma_e)
  int64_t n3;
  double* b;
  double* x;
  double* r;
  double* p;
  double* q;
  const double* dinv;
  double* red;  // 6 slots x gridDim.x
  int max_iter;
  double rtol;
  int* iters;
  double* res;
};

enum { kSlotMean = 0, kSlotPq = 1, kSlotRz = 2, kSlotRr = 3, kSlotBb = 4, kSlotX = 5, kNumSlots = 6 };

// Jacobi-preconditioned CG on the zero-mean subspace, x0 = 0.  Every loop
// is bounded by max_iter; all blocks take the same branch because they sum
// the same partials in the same order.
__global__ void __launch_bounds__(kEmgThreads) cg_kernel(CgArgs c) {
  cg::grid_group g = cg::this_grid();
  __shared__ double sh[kEmgThreads / 32];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // project b onto the zero-mean subspace (the compatible right-hand side)
  double s = 0.0;
  for (int64_t t = tid; t < c.n3; t += stride) s += c.b[t];
  block_partial(s, c.red, kSlotMean, sh);
  g.sync();
  const double mean_b = grid_total(c.red, kSlotMean, sh) / (double)c.n3;
  double rz = 0.0, bb = 0.0;
  for (int64_t t = tid; t < c.n3; t += stride) {
    const double bt = c.b[t] - mean_b;
    c.x[t] = 0.0;
    c.r[t] = bt;
    const double zt = bt * c.dinv[t];
    c.p[t] = zt;
    rz += bt * zt;
    bb += bt * bt;
  }
  block_partial(rz, c.red, kSlotRz, sh);
  block_partial(bb, c.red, kSlotBb, sh);
  g.sync();
  rz = grid_total(c.red, kSlotRz, sh);
  bb = grid_total(c.red, kSlotBb, sh);
  const double stop = c.rtol * c.rtol * bb;
  int it = 0;
  double rr = bb;
  while (it < c.max_iter && rr > stop && bb > 0.0) {
    double pq = 0.0;
    for (int64_t t = tid; t < c.n3; t += stride) {
      const double qt = apply_row(c.A, c.p, t);
      c.q[t] = qt;
      pq += c.p[t] * qt;
    }
    block_partial(pq, c.red, kSlotPq, sh);
    g.sync();
    pq = grid_total(c.red, kSlotPq, sh);
    const double alpha = pq > 0.0 ? rz / pq : 0.0;
    double rz_new = 0.0, rr_new = 0.0;
    for (int64_t t = tid; t < c.n3; t += stride) {
      c.x[t] += alpha * c.p[t];
      const double rt = c.r[t] - alpha * c.q[t];
      c.r[t] = rt;
      rz_new += rt * rt * c.dinv[t];
      rr_new += rt * rt;
    }
    block_partial(rz_new, c.red, kSlotRz, sh);
    block_partial(rr_new, c.red, kSlotRr, sh);
    g.sync();
    rz_new = grid_total(c.red, kSlotRz, sh);
    rr = grid_total(c.red, kSlotRr, sh);
    ++it;
    if (rr <= stop || pq <= 0.0) break;
    const double beta = rz > 0.0 ? rz_new / rz : 0.0;
    rz = rz_new;
    for (int64_t t = tid; t < c.n3; t += stride) c.p[t] = c.r[t] * c.dinv[t] + beta * c.p[t];
    g.sync();
  }
  // zero mean of the solution
  s = 0.0;
  for (int64_t t = tid; t < c.n3; t += stride) s += c.x[t];
  block_partial(s, c.red, kSlotX, sh);
  g.sync();
  const double mean_x = grid_total(c.red, kSlotX, sh) / (double)c.n3;
  for (int64_t t = tid; t < c.n3; t += stride) c.x[t] -= mean_x;
  if (tid == 0) {
    *c.iters = it;
    *c.res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

__global__ void to_float_kernel(const double* __restrict__ x, int64_t n, float* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)x[t];
}

fib_status emg_fail(fib_emg* e, fib_status s, const std::string& msg) {
  if (e) e->err = msg;
  return s;
}

#define EMG_CU(e, call)                                                                                  \
  do {                                                                                                   \
    cudaError_t err_ = (call);                                                                           \
    if (err_ != cudaSuccess)                                                                             \
      return emg_fail(e, err_ == cudaErrorMemoryAllocation ? FIB_ENOMEM : FIB_ECUDA,                     \
                      std::string(#call) + ": " + cudaGetErrorString(err_));                             \
  } while (0)

Stencil make_stencil(const fib_mesh3d& m, double sx, double sy, double sz) {
  Stencil s;
  s.nx = m.nx;
  s.ny = m.ny;
  s.nz = m.nz;
  s.hx = m.spacing[0];
  s.hy = m.spacing[1];
  s.hz = m.spacing[2];
  s.sx = sx;
  s.sy = sy;
  s.sz = sz;
  return s;
}

int grid_for(int64_t n, int threads) {
  const int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 65535));
}

void free_emg(fib_emg* e) {
  auto f = [](auto*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
  };
  f(e->d_rowptr);
  f(e->d_col);
  f(e->d_w);
  f(e->d_vm);
  f(e->d_v3);
  f(e->d_b);
  f(e->d_x);
  f(e->d_r);
  f(e->d_p);
  f(e->d_q);
  f(e->d_dinv);
  f(e->d_red);
  f(e->d_iters);
  f(e->d_res);
}

// Prolongation and right-hand side for the context's current V; leaves V3D
// in d_v3 and b in d_b.
fib_status prolongate_and_rhs(fib_emg* e, const fib::CtxView& v) {
  gather_ragged_kernel<<<grid_for(v.n_fibers, 1), 256, 0, v.stream>>>(v.fibers, v.n_fibers, v.u, e->d_vm, v.vrest);
  EMG_CU(e, cudaGetLastError());
  prolongate_kernel<<<grid_for(e->n3 * 32, kEmgThreads), kEmgThreads, 0, v.stream>>>(e->d_rowptr, e->d_col, e->d_w,
                                                                                      e->d_vm, e->n3, e->d_v3);
  EMG_CU(e, cudaGetLastError());
  *v.launches += 2;
  return FIB_OK;
}

}  // namespace

extern "C" {

fib_status fibers_emg_create(fib_ctx* ctx, const double* fiber_xy, double z0, const fib_mesh3d* mesh,
                             fib_emg** out) {
  if (!out) return FIB_EINVAL;
  *out = nullptr;
  fib::CtxView v;
  fib_status st = fib::ctx_view(ctx, &v);
  if (st != FIB_OK) return st;
  if (!mesh || (v.n_fibers > 0 && !fiber_xy))
    return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: mesh or fiber_xy is NULL");
  const fib_mesh3d& m = *mesh;
  if (m.reserved != 0) return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: mesh reserved field must be 0");
  if (m.nx < 2 || m.ny < 2 || m.nz < 2)
    return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: the 3D mesh needs at least 2 nodes per direction");
  for (int d = 0; d < 3; ++d)
    if (!(m.spacing[d] > 0.0) || !std::isfinite(m.spacing[d]) || !std::isfinite(m.origin[d]))
      return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: spacing must be > 0 and finite, origin finite");
  if (!(m.sigma_i >= 0.0) || !(m.sigma_e > 0.0) || !std::isfinite(m.sigma_i) || !std::isfinite(m.sigma_e))
    return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: need sigma_i >= 0 and sigma_e > 0, finite");
  const int64_t n3 = (int64_t)m.nx * m.ny * m.nz;
  if (n3 > ((int64_t)1 << 31)) return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: 3D mesh too large");
  if (v.total >= ((int64_t)1 << 31))
    return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: more than 2^31 fiber nodes");
  for (int32_t f = 0; f < v.n_fibers; ++f)
    if (!std::isfinite(fiber_xy[2 * f]) || !std::isfinite(fiber_xy[2 * f + 1]))
      return fib::ctx_fail(ctx, FIB_EINVAL, "fibers_emg_create: fiber position not finite");

  // eq:mapping_source_target: factors phi_t(xi_s) of every fiber node s for
  // the 8 nodes t of its element, then every row normalised by its sum
  const int64_t total = v.total;
  std::vector<int64_t> cnt(n3 + 1, 0);
  std::vector<int64_t> node_of(8 * (size_t)total);
  std::vector<double> fac(8 * (size_t)total);
  auto locate = [&](double p, int d, int n, int64_t* e, double* xi) {
    const double q = (p - m.origin[d]) / m.spacing[d];
    int64_t k = (int64_t)std::floor(q);
    k = std::min<int64_t>(std::max<int64_t>(k, 0), n - 2);
    *e = k;
    *xi = std::min(std::max(q - (double)k, 0.0), 1.0);
  };
  {
    int64_t s = 0;
    for (int32_t f = 0; f < v.n_fibers; ++f) {
      int64_t ex, ey;
      double xx, xy;
      locate(fiber_xy[2 * f], 0, m.nx, &ex, &xx);
      locate(fiber_xy[2 * f + 1], 1, m.ny, &ey, &xy);
      for (int32_t i = 0; i < v.n_nodes[f]; ++i, ++s) {
        int64_t ez;
        double xz;
        locate(z0 + v.h * (double)i, 2, m.nz, &ez, &xz);
        for (int c = 0; c < 8; ++c) {
          const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
          const double w = (cx ? xx : 1.0 - xx) * (cy ? xy : 1.0 - xy) * (cz ? xz : 1.0 - xz);
          const int64_t t = ((ez + cz) * m.ny + (ey + cy)) * m.nx + (ex + cx);
          node_of[8 * (size_t)s + c] = t;
          fac[8 * (size_t)s + c] = w;
          ++cnt[t + 1];
        }
      }
    }
  }
  std::vector<double> wsum(n3, 0.0);
  for (size_t q = 0; q < node_of.size(); ++q) wsum[node_of[q]] += fac[q];
  std::vector<int64_t> rowptr(n3 + 1, 0);
  for (int64_t t = 0; t < n3; ++t) rowptr[t + 1] = rowptr[t] + cnt[t + 1];
  std::vector<int64_t> fill(rowptr.begin(), rowptr.end() - 1);
  std::vector<int32_t> col(8 * (size_t)total);
  std::vector<float> wgt(8 * (size_t)total);
  // points in ragged order, so each row's columns come out ascending
  for (int64_t s = 0; s < total; ++s)
    for (int c = 0; c < 8; ++c) {
      const int64_t t = node_of[8 * (size_t)s + c];
      const int64_t q = fill[t]++;
      col[q] = (int32_t)s;
      wgt[q] = wsum[t] > 0.0 ? (float)(fac[8 * (size_t)s + c] / wsum[t]) : 0.0f;
    }

  fib_emg* e = new (std::nothrow) fib_emg();
  if (!e) return fib::ctx_fail(ctx, FIB_ENOMEM, "fibers_emg_create: host allocation failed");
  e->fibers = ctx;
  e->device = v.device;
  e->stream = v.stream;
  e->mesh = m;
  e->n3 = n3;
  e->n_pts = total;
  auto fail = [&](fib_status s2, const char* what, cudaError_t ce) {
    std::string msg = std::string("fibers_emg_create: ") + what + ": " + cudaGetErrorString(ce);
    free_emg(e);
    delete e;
    return fib::ctx_fail(ctx, s2, msg.c_str());
  };
  cudaError_t ce = cudaSetDevice(v.device);
  if (ce != cudaSuccess) return fail(FIB_ECUDA, "set device", ce);
  const size_t nnz = col.size();
#define EMG_ALLOC(ptr, bytes)                                                                            \
  if ((ce = cudaMalloc(&(ptr), std::max<size_t>((bytes), 16))) != cudaSuccess)                            \
    return fail(ce == cudaErrorMemoryAllocation ? FIB_ENOMEM : FIB_ECUDA, "allocation", ce);
  EMG_ALLOC(e->d_rowptr, sizeof(int64_t) * (n3 + 1));
  EMG_ALLOC(e->d_col, sizeof(int32_t) * nnz);
  EMG_ALLOC(e->d_w, sizeof(float) * nnz);
  EMG_ALLOC(e->d_vm, sizeof(float) * total);
  EMG_ALLOC(e->d_v3, sizeof(double) * n3);
  EMG_ALLOC(e->d_b, sizeof(double) * n3);
  EMG_ALLOC(e->d_x, sizeof(double) * n3);
  EMG_ALLOC(e->d_r, sizeof(double) * n3);
  EMG_ALLOC(e->d_p, sizeof(double) * n3);
  EMG_ALLOC(e->d_q, sizeof(double) * n3);
  EMG_ALLOC(e->d_dinv, sizeof(double) * n3);
  EMG_ALLOC(e->d_iters, sizeof(int));
  EMG_ALLOC(e->d_res, sizeof(double));
#undef EMG_ALLOC
  // cooperative grid: every block must be resident at once
  int per_sm = 0, n_sm = 0;
  if ((ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel, kEmgThreads, 0)) != cudaSuccess)
    return fail(FIB_ECUDA, "occupancy", ce);
  if ((ce = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, v.device)) != cudaSuccess)
    return fail(FIB_ECUDA, "device attribute", ce);
  int coop = 0;
  if ((ce = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, v.device)) != cudaSuccess)
    return fail(FIB_ECUDA, "device attribute", ce);
  if (!coop || per_sm < 1) {
    free_emg(e);
    delete e;
    return fib::ctx_fail(ctx, FIB_ENOTSUP, "fibers_emg_create: the device has no cooperative launch");
  }
  e->grid = (int)std::min<int64_t>((int64_t)per_sm * n_sm, (n3 + kEmgThreads - 1) / kEmgThreads);
  e->grid = std::max(e->grid, 1);
  if ((ce = cudaMalloc(&e->d_red, sizeof(double) * kNumSlots * (size_t)e->grid)) != cudaSuccess)
    return fail(FIB_ENOMEM, "allocation", ce);
  if ((ce = cudaMemcpy(e->d_rowptr, rowptr.data(), sizeof(int64_t) * (n3 + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (nnz > 0 && (ce = cudaMemcpy(e->d_col, col.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice)) !=
                      cudaSuccess) ||
      (nnz > 0 && (ce = cudaMemcpy(e->d_w, wgt.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice)) != cudaSuccess))
    return fail(FIB_ECUDA, "upload", ce);
  const Stencil At = make_stencil(m, m.sigma_e, m.sigma_e, m.sigma_i + m.sigma_e);
  diag_kernel<<<grid_for(n3, 256), 256, 0, e->stream>>>(At, n3, e->d_dinv);
  if ((ce = cudaGetLastError()) != cudaSuccess) return fail(FIB_ECUDA, "diagonal kernel", ce);
  if ((ce = cudaStreamSynchronize(e->stream)) != cudaSuccess) return fail(FIB_ECUDA, "setup", ce);
  ++*v.launches;
  *out = e;
  return FIB_OK;
}

fib_status fibers_emg_vm3d(fib_emg* e, double* out, size_t capacity, int32_t out_is_device) {
  if (!e) return FIB_EINVAL;
  fib::CtxView v;
  fib_status st = fib::ctx_view(e->fibers, &v);
  if (st != FIB_OK) return st;
  if (capacity < (size_t)e->n3 || !out) return emg_fail(e, FIB_EINVAL, "capacity < 3D nodes or out is NULL");
  EMG_CU(e, cudaSetDevice(e->device));
  st = prolongate_and_rhs(e, v);
  if (st != FIB_OK) return st;
  EMG_CU(e, cudaMemcpyAsync(out, e->d_v3, sizeof(double) * e->n3,
                            out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->stream));
  EMG_CU(e, cudaStreamSynchronize(e->stream));
  return FIB_OK;
}

fib_status fibers_emg_phi_e(fib_emg* e, float* out, size_t capacity, int32_t out_is_device, double rtol,
                            int32_t max_iter, int32_t* iterations, double* rel_residual) {
  if (!e) return FIB_EINVAL;
  fib::CtxView v;
  fib_status st = fib::ctx_view(e->fibers, &v);
  if (st != FIB_OK) return st;
  if (capacity < (size_t)e->n3 || !out) return emg_fail(e, FIB_EINVAL, "capacity < 3D nodes or out is NULL");
  if (!(rtol > 0.0) || !std::isfinite(rtol) || max_iter < 1)
    return emg_fail(e, FIB_EINVAL, "need rtol > 0 and max_iter >= 1");
  EMG_CU(e, cudaSetDevice(e->device));
  st = prolongate_and_rhs(e, v);
  if (st != FIB_OK) return st;
  const fib_mesh3d& m = e->mesh;
  const Stencil Si = make_stencil(m, 0.0, 0.0, m.sigma_i);
  rhs_kernel<<<grid_for(e->n3, 256), 256, 0, e->stream>>>(Si, e->d_v3, e->n3, e->d_b);
  EMG_CU(e, cudaGetLastError());
  CgArgs a;
  a.A = make_stencil(m, m.sigma_e, m.sigma_e, m.sigma_i + m.sigma_e);
  a.n3 = e->n3;
  a.b = e->d_b;
  a.x = e->d_x;
  a.r = e->d_r;
  a.p = e->d_p;
  a.q = e->d_q;
  a.dinv = e->d_dinv;
  a.red = e->d_red;
  a.max_iter = max_iter;
  a.rtol = rtol;
  a.iters = e->d_iters;
  a.res = e->d_res;
  void* args[] = {&a};
  EMG_CU(e, cudaLaunchCooperativeKernel((const void*)cg_kernel, dim3(e->grid), dim3(kEmgThreads), args, 0,
                                        e->stream));
  float* dst = out;
  if (!out_is_device) dst = reinterpret_cast<float*>(e->d_q);  // q is free after the solve: stage the floats there
  to_float_kernel<<<grid_for(e->n3, 256), 256, 0, e->stream>>>(e->d_x, e->n3, dst);
  EMG_CU(e, cudaGetLastError());
  *v.launches += 3;
  if (!out_is_device) EMG_CU(e, cudaMemcpyAsync(out, dst, sizeof(float) * e->n3, cudaMemcpyDeviceToHost, e->stream));
  int it = 0;
  double res = 0.0;
  EMG_CU(e, cudaMemcpyAsync(&it, e->d_iters, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
  EMG_CU(e, cudaMemcpyAsync(&res, e->d_res, sizeof(double), cudaMemcpyDeviceToHost, e->stream));
  EMG_CU(e, cudaStreamSynchronize(e->stream));
  if (iterations) *iterations = it;
  if (rel_residual) *rel_residual = res;
  if (!(res <= rtol)) return emg_fail(e, FIB_ETIMEOUT, "conjugate gradients did not reach rtol in max_iter");
  return FIB_OK;
}

int64_t fibers_emg_nodes(const fib_emg* e) { return e ? e->n3 : 0; }

const char* fibers_emg_last_error(const fib_emg* e) { return e ? e->err.c_str() : ""; }

void fibers_emg_destroy(fib_emg* e) {
  if (!e) return;
  cudaSetDevice(e->device);
  if (e->stream) cudaStreamSynchronize(e->stream);
  free_emg(e);
  delete e;
}

}  // extern "C"
