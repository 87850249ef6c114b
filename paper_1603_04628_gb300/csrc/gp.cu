// Gaussian-process surrogate on the GPU, FP64 throughout (paper Sec. 2.2):
//   - Eq. d2Eq scales: mean pairwise separation of the database inputs per
//     dimension (recomputed at every fit);
//   - Eq. quadraticKernelEq + Eq. covarianceEq: C = K(X, X) + sn2 I;
//   - blocked right-looking Cholesky C = L L^T (32 x 32 tiles);
//   - alpha = C^-1 (y - mu(X)) by forward and backward substitution;
//   - Eq. predMeanEq / predVarEq: per query, k* = K(x*, X), mean =
//     mu(x*) + k*.alpha, v = L^-1 k*, var = sf2 - |v|^2 (latent variance,
//     clamped at zero), fused into one kernel per query.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mdgp.h"
#include "md_ctx.h"

namespace {

constexpr int TB = 32;            // Cholesky tile
constexpr int kMaxD = 8;          // input dimensions supported
constexpr int kMaxM = 16384;      // database entries supported (predict keeps v in shared memory)
constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

// Row sums of the pair separations: rows[i D + k] = sum over j > i of
// |x_ik - x_jk|.  Block i takes row i, its threads stride over j > i; the
// sums meet in a fixed order, so the scales do not depend on scheduling.
__global__ void k_gp_pairsep(const double* X, int M, int D, double* rows) {
  __shared__ double part[kMaxD][32];
  const int i = blockIdx.x;
  double xi[kMaxD], acc[kMaxD];
  for (int k = 0; k < D; ++k) { xi[k] = X[(size_t)i * D + k]; acc[k] = 0.0; }
  for (int j = i + 1 + threadIdx.x; j < M; j += blockDim.x)
    for (int k = 0; k < D; ++k) acc[k] += fabs(xi[k] - X[(size_t)j * D + k]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < D; ++k) {
    const double s = warp_sum_d(acc[k]);
    if (lane == 0) part[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < D) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[threadIdx.x][w];
    rows[(size_t)i * D + threadIdx.x] = s;
  }
}

// Per-dimension scale used where the mean separation is undefined.
struct Fallback {
  double v[kMaxD];
};

static Fallback make_fallback(const mdgp_gp_params* p, int D) {
  Fallback f;
  const double one = p->fallback_scale > 0 ? p->fallback_scale : 1.0;
  for (int k = 0; k < kMaxD; ++k) f.v[k] = one;
  if (p->fallback_scales)
    for (int k = 0; k < D; ++k)
      if (p->fallback_scales[k] > 0) f.v[k] = p->fallback_scales[k];
  return f;
}

// Scales of Eq. d2Eq: the mean separation over all pairs i < j of each
// dimension (the row sums of k_gp_pairsep added in a fixed order), or the
// fallback where it is undefined (M < 2 or no spread), or the fixed scales.
// One block.
__global__ void k_gp_scales(const double* rows, double* scale, int M, int D, Fallback fallback,
                            const double* fixed) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < D; ++k) {
    double s = 0.0;
    if (!fixed)
      for (int i = threadIdx.x; i < M; i += blockDim.x) s += rows[(size_t)i * D + k];
    s = warp_sum_d(s);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      double v = fallback.v[k];
      if (fixed) {
        v = fixed[k];
      } else if (M >= 2) {
        const double m = t / (0.5 * (double)M * (double)(M - 1));
        if (m > 0.0) v = m;
      }
      scale[k] = v;
    }
    __syncthreads();
  }
}

// The covariance function.  Squared exponential (Eq. quadraticKernelEq) on
// the inputs scaled by Eq. d2Eq, or, when the first scale is negative, the
// periodic kernel of App. B (Eq. periodicKernel) on one input with period
// -scale[0]: sf2 exp(-2 sin^2(pi |t - t'| / T) / l2).
__device__ __forceinline__ double se_kernel(const double* a, const double* b, const double* scale, int D,
                                            double sf2, double l2) {
  if (scale[0] < 0.0) {
    const double sn = sinpi(fabs(a[0] - b[0]) / -scale[0]);
    return sf2 * exp(-2.0 * sn * sn / l2);
  }
  double d2 = 0.0;
  for (int k = 0; k < D; ++k) {
    const double t = (a[k] - b[k]) / scale[k];
    d2 += t * t;
  }
  return sf2 * exp(-d2 / (2.0 * l2));
}

// C (Mp x Mp, row-major, lower part used): K + sn2 I, identity on the padding.
__global__ void k_gp_cov(const double* X, int M, int Mp, int D, const double* scale, double sf2, double l2,
                         double sn2, double* C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= Mp) return;
  double v;
  if (i < M && j < M) {
    v = se_kernel(X + (size_t)i * D, X + (size_t)j * D, scale, D, sf2, l2);
    if (i == j) v += sn2;
  } else {
    v = (i == j) ? 1.0 : 0.0;
  }
  C[(size_t)i * Mp + j] = v;
}

// Cholesky of the diagonal tile kb in place (lower), four warps: the tile
// sits in shared memory, lane i of every warp works on row i, and warp w owns
// the columns c = w (mod 4), so that the right-looking updates of each step
// run on all four FP64 pipes of the SM (one warp would leave three idle, and
// FP64 issues at 1/64 of the FP32 rate here).  Step k: the owner of column k
// has scaled it (pivot p = d rsqrt(d), column times rsqrt(d)); after a block
// barrier every warp applies T[i][c] -= T[i][k] T[c][k] to its columns c > k,
// the owner of column k + 1 first, which then takes the next pivot and scales
// its column while the others are still updating.  Each element receives its
// updates in the order of k, as in the one-warp form.  A non-positive pivot
// sets *status.
__device__ __forceinline__ void potrf_pivot(double (*T)[TB + 1], int k, int i, int* status) {   // whole warp
  const double d = T[k][k];
  __syncwarp();   // every lane has read the pivot before lane k overwrites it
  const bool ok = d > 0.0;
  if (i == k && !ok) atomicMin(status, MDGP_E_NOTPD);
  const double dd = ok ? d : 1e-300;
  const double rp = rsqrt(dd);   // one FP64 routine instead of sqrt and a divide
  if (i == k) T[k][k] = dd * rp;
  if (i > k) T[i][k] *= rp;
}

__global__ void __launch_bounds__(4 * TB) k_potrf_diag(double* A, int Mp, int kb, int* status) {
  __shared__ double T[TB][TB + 1];
  const int i = threadIdx.x & (TB - 1), w = threadIdx.x >> 5;
  const size_t base = (size_t)kb * TB;
  for (int c = w; c < TB; c += 4) T[i][c] = A[(base + i) * Mp + base + c];
  __syncthreads();
  if (w == 0) potrf_pivot(T, 0, i, status);
  for (int k = 0; k < TB - 1; ++k) {
    __syncthreads();   // column k scaled
    const double tik = T[i][k];
    // the owner of column k + 1 updates it first and takes the next pivot
    if (w == ((k + 1) & 3)) {
      if (i >= k + 1) T[i][k + 1] -= tik * T[k + 1][k];
      __syncwarp();
      potrf_pivot(T, k + 1, i, status);
    }
    for (int c = (k + 2) + ((w - (k + 2)) & 3); c < TB; c += 4)
      if (i >= c) T[i][c] -= tik * T[c][k];
  }
  __syncthreads();
  for (int c = w; c < TB; c += 4) A[(base + i) * Mp + base + c] = c <= i ? T[i][c] : 0.0;
}

// Panel: A_ik <- A_ik L_kk^-T for every tile row i > kb.  A block of
// TB x kTrsmRows threads takes kTrsmRows rows of one tile (TB / kTrsmRows
// blocks per tile, so early panels spread over more SMs).  Each row solves
// x L^T = a; the block sweeps the columns: once x_j is final (times 1/L_jj)
// every later column c subtracts x_j L_cj, rows and columns in parallel.
constexpr int kTrsmRows = 8;

__global__ void k_trsm_panel(double* A, int Mp, int kb) {
  __shared__ double L[TB][TB + 1];
  __shared__ double X[kTrsmRows][TB + 1];
  __shared__ double rd[TB];
  const int r = threadIdx.y, c = threadIdx.x;
  constexpr int parts = TB / kTrsmRows;
  const int ib = kb + 1 + blockIdx.x / parts;
  const int r_off = (blockIdx.x % parts) * kTrsmRows;
  const size_t kr = (size_t)kb * TB, ir = (size_t)ib * TB + r_off;
  for (int rr = r; rr < TB; rr += kTrsmRows) L[rr][c] = A[(kr + rr) * Mp + kr + c];
  X[r][c] = A[(ir + r) * Mp + kr + c];
  __syncthreads();
  if (r == 0) rd[c] = 1.0 / L[c][c];
  __syncthreads();
  for (int j = 0; j < TB; ++j) {
    if (c == j) X[r][j] *= rd[j];
    __syncthreads();
    if (c > j) X[r][c] -= X[r][j] * L[c][j];
    __syncthreads();
  }
  A[(ir + r) * Mp + kr + c] = X[r][c];
}

// Trailing update: A_ij -= L_ik L_jk^T (one block per tile) for the tiles
// kb < j <= i (part 0), the next tile column j = kb + 1 alone (part 1), or
// the tiles kb + 1 < j <= i (part 2); parts 1 and 2 together are part 0.
__global__ void k_syrk_update(double* A, int Mp, int kb, int nt, int part) {
  __shared__ double Li[TB][TB + 1];
  __shared__ double Lj[TB][TB + 1];
  // map blockIdx.x to a lower-triangle tile (i, j) of the trailing matrix
  int i = 0, j = 0;
  if (part == 1) {
    i = blockIdx.x;
  } else {
    int t = blockIdx.x;
    while (t > i) { t -= i + 1; ++i; }
    j = t;
    if (part == 2) { ++i; ++j; }
  }
  const int ib = kb + 1 + i, jb = kb + 1 + j;
  if (ib >= nt) return;
  const int r = threadIdx.y, c = threadIdx.x;
  const size_t kr = (size_t)kb * TB;
  Li[r][c] = A[((size_t)ib * TB + r) * Mp + kr + c];
  Lj[r][c] = A[((size_t)jb * TB + r) * Mp + kr + c];
  __syncthreads();
  double s = 0.0;
#pragma unroll 8
  for (int l = 0; l < TB; ++l) s += Li[r][l] * Lj[c][l];
  A[((size_t)ib * TB + r) * Mp + (size_t)jb * TB + c] -= s;
}

// alpha = C^-1 (y - mu) by blocked forward then backward substitution in one
// block (the allocation-free entry point's solve: one launch, no work
// buffer; fits use the tile-column launches below).  Forward (L z = r), tile
// row by tile row: warp w
// subtracts from z of row r0 + w its dot product with the solved part (lanes
// over the row: coalesced), the TB x TB diagonal tile is staged in shared
// memory and warp 0 solves the triangle.  Backward (L^T a = z): lane i owns
// row r0 + i and the warps split the solved rows below (lanes read one row of
// L: coalesced), the partial sums meet in shared memory, then warp 0 solves
// the transposed triangle.
__global__ void __launch_bounds__(1024) k_gp_alpha(const double* L, int M, int Mp, const double* y,
                                                   const double* mu, double* alpha, double* r_dot_alpha) {
  extern __shared__ double z[];
  __shared__ double T[TB][TB + 1];
  __shared__ double part[32][TB + 1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < Mp; i += nt) z[i] = i < M ? y[i] - (mu ? mu[i] : 0.0) : 0.0;
  __syncthreads();
  const int nblk = Mp / TB;
  for (int kb = 0; kb < nblk; ++kb) {
    const int r0 = kb * TB;
    for (int rr = wid; rr < TB; rr += nw) {
      const int row = r0 + rr;
      double s = 0.0;
      for (int j = lane; j < r0; j += 32) s += L[(size_t)row * Mp + j] * z[j];
      s = warp_sum_d(s);
      T[rr][lane] = L[(size_t)row * Mp + r0 + lane];
      if (lane == 0) z[row] -= s;
    }
    __syncthreads();
    if (wid == 0) {
      double x = z[r0 + lane];
      const double rdl = 1.0 / T[lane][lane];
      for (int j = 0; j < TB; ++j) {
        if (lane == j) x *= rdl;
        const double xs = __shfl_sync(kFullMask, x, j);
        if (lane > j) x -= T[lane][j] * xs;
      }
      z[r0 + lane] = x;
    }
    __syncthreads();
  }
  for (int kb = nblk - 1; kb >= 0; --kb) {
    const int r0 = kb * TB;
    double s = 0.0;
    for (int j = r0 + TB + wid; j < Mp; j += nw) s += L[(size_t)j * Mp + r0 + lane] * z[j];
    part[wid][lane] = s;
    for (int rr = wid; rr < TB; rr += nw) T[rr][lane] = L[(size_t)(r0 + rr) * Mp + r0 + lane];
    __syncthreads();
    if (wid == 0) {
      double tot = 0.0;
      for (int w = 0; w < nw; ++w) tot += part[w][lane];
      double x = z[r0 + lane] - tot;
      const double rdl = 1.0 / T[lane][lane];
      for (int j = TB - 1; j >= 0; --j) {
        if (lane == j) x *= rdl;
        const double xs = __shfl_sync(kFullMask, x, j);
        if (lane < j) x -= T[j][lane] * xs;
      }
      z[r0 + lane] = x;
    }
    __syncthreads();
  }
  for (int i = tid; i < M; i += nt) alpha[i] = z[i];
  if (r_dot_alpha) {
    // (y - mu)^T alpha, the data term of Eq. evidenceEq
    double s = 0.0;
    for (int i = tid; i < M; i += nt) s += (y[i] - (mu ? mu[i] : 0.0)) * z[i];
    s = warp_sum_d(s);
    __syncthreads();
    if (lane == 0) part[wid][0] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += part[w][0];
      *r_dot_alpha = t;
    }
  }
}

// alpha = C^-1 (y - mu) over many SMs: one launch per tile column, forward
// (L z = r) then backward (L^T a = z).  In the launch for tile kb every block
// stages the diagonal tile and solves it (its right-hand side is final: the
// launches for the earlier tiles have subtracted their parts), block 0
// stores the TB unknowns, and the grid subtracts their contribution from the
// unknowns still open.  The unknowns of tile kb are read only in its own
// launch and every open unknown is updated by one thread, so the launches
// need no synchronisation beyond their order on the stream.
//
// Forward, tile kb: z_kb from r_kb, then r_i -= sum_c L_{i, kb TB + c} z_c
// for the rows i below the tile, one warp per row (lanes along the row).
__global__ void __launch_bounds__(256) k_tri_fwd(const double* L, int Mp, int kb, double* r, double* z) {
  __shared__ double T[TB][TB + 1];
  __shared__ double zt[TB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r0 = kb * TB;
  for (int rr = wid; rr < TB; rr += nw) T[rr][lane] = L[(size_t)(r0 + rr) * Mp + r0 + lane];
  __syncthreads();
  if (wid == 0) {
    double x = r[r0 + lane];
    const double rdl = 1.0 / T[lane][lane];
    for (int j = 0; j < TB; ++j) {
      if (lane == j) x *= rdl;
      const double xs = __shfl_sync(kFullMask, x, j);
      if (lane > j) x -= T[lane][j] * xs;
    }
    zt[lane] = x;
    if (blockIdx.x == 0) z[r0 + lane] = x;
  }
  __syncthreads();
  for (int i = r0 + TB + blockIdx.x * nw + wid; i < Mp; i += gridDim.x * nw) {
    const double t = warp_sum_d(L[(size_t)i * Mp + r0 + lane] * zt[lane]);
    if (lane == 0) r[i] -= t;
  }
}

// Backward, tile kb: a_kb from t_kb (the transposed diagonal tile), then
// t_i -= sum_c L_{kb TB + c, i} a_c for the unknowns i above the tile, one
// thread per i (consecutive threads read consecutive columns).
__global__ void __launch_bounds__(256) k_tri_bwd(const double* L, int Mp, int kb, double* t, double* a) {
  __shared__ double T[TB][TB + 1];
  __shared__ double at[TB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r0 = kb * TB;
  for (int rr = wid; rr < TB; rr += nw) T[rr][lane] = L[(size_t)(r0 + rr) * Mp + r0 + lane];
  __syncthreads();
  if (wid == 0) {
    double x = t[r0 + lane];
    const double rdl = 1.0 / T[lane][lane];
    for (int j = TB - 1; j >= 0; --j) {
      if (lane == j) x *= rdl;
      const double xs = __shfl_sync(kFullMask, x, j);
      if (lane < j) x -= T[j][lane] * xs;
    }
    at[lane] = x;
    if (blockIdx.x == 0) a[r0 + lane] = x;
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r0; i += gridDim.x * blockDim.x) {
    double sum = 0.0;
#pragma unroll 8
    for (int c = 0; c < TB; ++c) sum += L[(size_t)(r0 + c) * Mp + i] * at[c];
    t[i] -= sum;
  }
}

// r = y - mu on the M data rows, 0 on the padding (Mp).
__global__ void k_gp_resid(const double* y, const double* mu, int M, int Mp, double* r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Mp) r[i] = i < M ? y[i] - (mu ? mu[i] : 0.0) : 0.0;
}

// (y - mu)^T alpha, the data term of Eq. evidenceEq (one block).
__global__ void k_gp_dot(const double* y, const double* mu, const double* alpha, int M, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) s += (y[i] - (mu ? mu[i] : 0.0)) * alpha[i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    *out = tot;
  }
}

// sum_i log L_ii over the M data rows: half the log-determinant of C
// (Eq. evidenceEq).
__global__ void k_gp_logdiag(const double* L, int M, int Mp, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) s += log(L[(size_t)i * Mp + i]);
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// One query per block: k*, mean, v = L^-1 k* by blocked forward
// substitution (tile rows of TB: a warp per row subtracts the solved part,
// then one warp solves the TB x TB triangle from shared memory),
// var = sf2 - |v|^2.  Without with_var the block stops after the mean.
__global__ void k_gp_predict(const double* X, const double* L, const double* alpha, const double* scale,
                             int M, int Mp, int D, double sf2, double l2, const double* Xs, const double* mus,
                             double* mean, double* var, bool with_var) {
  extern __shared__ double v[];
  __shared__ double xq[kMaxD];
  __shared__ double red[32];
  __shared__ double T[TB][TB + 1];
  const int q = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  if (tid < D) xq[tid] = Xs[(size_t)q * D + tid];
  __syncthreads();
  double dot = 0.0;
  for (int i = tid; i < Mp; i += nt) {
    const double k = i < M ? se_kernel(xq, X + (size_t)i * D, scale, D, sf2, l2) : 0.0;
    v[i] = k;
    if (i < M && alpha) dot += k * alpha[i];
  }
  dot = warp_sum_d(dot);
  if (lane == 0) red[wid] = dot;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t += red[w];
    mean[q] = (mus ? mus[q] : 0.0) + t;
  }
  __syncthreads();
  if (!with_var) return;
  const int nblk = Mp / TB, nw = nt >> 5;
  for (int kb = 0; kb < nblk; ++kb) {
    // rows of tile kb minus the solved part, v_r -= sum_{j < kb*TB} L_rj v_j:
    // one warp per row, lanes along the row (coalesced); the diagonal tile
    // goes to shared memory for the triangle
    const int r0 = kb * TB;
    for (int rr = wid; rr < TB; rr += nw) {
      const int row = r0 + rr;
      double s = 0.0;
      for (int j = lane; j < r0; j += 32) s += L[(size_t)row * Mp + j] * v[j];
      s = warp_sum_d(s);
      T[rr][lane] = L[(size_t)row * Mp + r0 + lane];
      if (lane == 0) v[row] -= s;
    }
    __syncthreads();
    // triangle solve by warp 0: lane r owns row r0 + r
    if (wid == 0) {
      double x = v[r0 + lane];
      const double rdl = 1.0 / T[lane][lane];
      for (int j = 0; j < TB; ++j) {
        if (lane == j) x *= rdl;
        const double xs = __shfl_sync(kFullMask, x, j);   // solved unknown j
        if (lane > j) x -= T[lane][j] * xs;
      }
      v[r0 + lane] = x;
    }
    __syncthreads();
  }
  double ss = 0.0;
  for (int i = tid; i < M; i += nt) ss += v[i] * v[i];
  ss = warp_sum_d(ss);
  if (lane == 0) red[wid] = ss;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t += red[w];
    const double vv = sf2 - t;
    var[q] = vv > 0.0 ? vv : 0.0;
  }
}

}  // namespace

// The solve kernels keep one vector of Mp doubles in dynamic shared memory.
// Every path sets their limit to the largest database (kMaxM entries) before
// it launches them, never to less: the limit belongs to the kernel, so a
// smaller value set for one call would make a later, larger launch fail.
static cudaError_t allow_solve_smem() {
  constexpr int kSolveSmem = kMaxM * (int)sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_gp_alpha, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  return e;
}

struct mdgp_gp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int M = 0, Mp = 0, D = 0;
  double sf2 = 1, l2 = 1, sn2 = 0;
  double period = 0;   // > 0: the periodic kernel of App. B
  double *dX = nullptr, *dL = nullptr, *dalpha = nullptr, *dscale = nullptr;
  double* dwork = nullptr;   // 2 Mp: right-hand side and forward solution of the alpha solve
  double *dq = nullptr, *dmu = nullptr, *dmean = nullptr, *dvar = nullptr;
  size_t qcap = 0;
  bool has_alpha = true;   // false: factor only (posterior variances, no means or evidence)
  cudaStream_t fs[2] = {nullptr, nullptr};   // lookahead streams and events of the context (fit only)
  cudaEvent_t fe[4] = {nullptr, nullptr, nullptr, nullptr};
  int launches = 0;
  char err[128] = {0};
};

static int gp_err(mdgp_gp* g, cudaError_t e) {
  if (e == cudaSuccess) return MDGP_OK;
  if (g) std::snprintf(g->err, sizeof(g->err), "%s", cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MDGP_E_NOMEM : MDGP_E_CUDA;
}

#define GK(expr)                                  \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return gp_err(g, e_);  \
  } while (0)

static void gp_release(mdgp_gp* g) {
  for (double** p : {&g->dX, &g->dL, &g->dalpha, &g->dscale, &g->dwork, &g->dq, &g->dmu, &g->dmean, &g->dvar})
    if (*p) { cudaFree(*p); *p = nullptr; }
}

// Blocked Cholesky with a lookahead of one tile column.  The trailing update
// of step k is split: its next tile column (k + 1) stays on the chain stream
// with the diagonal factorisation and the panel solve, the rest of it runs
// on a second, lower-priority stream and overlaps the next step's diagonal
// tile and panel.  The next column update waits for the previous bulk update
// (the same tiles), so every tile receives its updates in the order of k and
// the factor is the one the single-stream loop computes, bit for bit.
constexpr int kLookaheadTiles = 4;

static int enqueue_cholesky_lookahead(mdgp_gp* g, int* dstatus) {
  const int Mp = g->Mp, nt = Mp / TB;
  cudaStream_t s = g->stream, sa = g->fs[0], sb = g->fs[1];
  cudaEvent_t e_in = g->fe[0], e_panel = g->fe[1], e_bulk = g->fe[2], e_out = g->fe[3];
  GK(cudaEventRecord(e_in, s));   // the covariance is built on s
  GK(cudaStreamWaitEvent(sa, e_in, 0));
  GK(cudaStreamWaitEvent(sb, e_in, 0));
  for (int kb = 0; kb < nt; ++kb) {
    k_potrf_diag<<<1, 4 * TB, 0, sa>>>(g->dL, Mp, kb, dstatus);
    g->launches++;
    const int rest = nt - kb - 1;
    if (rest == 0) break;
    k_trsm_panel<<<rest * (TB / kTrsmRows), dim3(TB, kTrsmRows), 0, sa>>>(g->dL, Mp, kb);
    GK(cudaEventRecord(e_panel, sa));
    if (kb > 0) GK(cudaStreamWaitEvent(sa, e_bulk, 0));   // bulk update of step kb - 1
    k_syrk_update<<<rest, dim3(TB, TB), 0, sa>>>(g->dL, Mp, kb, nt, 1);
    g->launches += 2;
    if (rest > 1) {
      GK(cudaStreamWaitEvent(sb, e_panel, 0));
      k_syrk_update<<<rest * (rest - 1) / 2, dim3(TB, TB), 0, sb>>>(g->dL, Mp, kb, nt, 2);
      GK(cudaEventRecord(e_bulk, sb));
      g->launches++;
    }
  }
  GK(cudaEventRecord(e_out, sb));
  GK(cudaStreamWaitEvent(s, e_out, 0));
  GK(cudaEventRecord(e_out, sa));
  GK(cudaStreamWaitEvent(s, e_out, 0));
  return MDGP_OK;
}

// alpha = C^-1 (y - mu) on the factor, (y - mu)^T alpha and sum log L_ii
// for the evidence (dy, dmu: M device values; dmu nullable).
static int enqueue_alpha(mdgp_gp* g, const double* dy, const double* dmu) {
  const int M = g->M, Mp = g->Mp;
  cudaStream_t s = g->stream;
  const int nt = Mp / TB;
  double *r = g->dwork, *z = g->dwork + Mp;
  k_gp_resid<<<(Mp + 255) / 256, 256, 0, s>>>(dy, dmu, M, Mp, r);
  for (int kb = 0; kb < nt; ++kb) {
    const int rows = Mp - (kb + 1) * TB;                 // rows below the tile, 8 per block
    const int blocks = rows > 0 ? (rows + 7) / 8 : 1;
    k_tri_fwd<<<blocks, 256, 0, s>>>(g->dL, Mp, kb, r, z);
  }
  for (int kb = nt - 1; kb >= 0; --kb) {
    const int cols = kb * TB;                            // unknowns above the tile, 256 per block
    const int blocks = cols > 0 ? (cols + 255) / 256 : 1;
    k_tri_bwd<<<blocks, 256, 0, s>>>(g->dL, Mp, kb, z, g->dalpha);
  }
  k_gp_dot<<<1, 1024, 0, s>>>(dy, dmu, g->dalpha, M, g->dscale + kMaxD);
  k_gp_logdiag<<<1, 256, 0, s>>>(g->dL, M, Mp, g->dscale + kMaxD + 1);
  g->launches += 2 * nt + 3;
  return MDGP_OK;
}

static int gp_fit_impl(mdgp_gp* g, const double* X, const double* y, const double* mu_X,
                       const mdgp_gp_params* p) {
  const int M = g->M, D = g->D, Mp = g->Mp;
  cudaStream_t s = g->stream;
  // the scales, then (y - mu)^T alpha and sum log L_ii for the evidence
  GK(cudaMalloc(&g->dscale, sizeof(double) * (kMaxD + 2)));
  GK(cudaMemsetAsync(g->dscale, 0, sizeof(double) * (kMaxD + 2), s));
  // the periodic kernel takes no scales: its first scale carries -period
  const double neg_period = -p->period;
  const double* fixed = p->period > 0.0 ? &neg_period : p->fixed_scales;
  if (M == 0) {
    const Fallback f = make_fallback(p, D);
    std::vector<double> fb(f.v, f.v + D);
    if (p->period > 0.0) fb[0] = neg_period;
    GK(cudaMemcpyAsync(g->dscale, fb.data(), sizeof(double) * D, cudaMemcpyHostToDevice, s));
    GK(cudaStreamSynchronize(s));
    return MDGP_OK;
  }
  // the fit's own scratch, freed on every way out (error returns included;
  // cudaFree waits for the work still queued on it)
  struct Scratch {
    double *dy = nullptr, *dmuX = nullptr, *dfixed = nullptr;
    int* dstatus = nullptr;
    ~Scratch() {
      if (dy) cudaFree(dy);
      if (dstatus) cudaFree(dstatus);
      if (dmuX) cudaFree(dmuX);
      if (dfixed) cudaFree(dfixed);
    }
  } sc;
  double*& dy = sc.dy;
  double*& dmuX = sc.dmuX;
  double*& dfixed = sc.dfixed;
  int*& dstatus = sc.dstatus;
  GK(cudaMalloc(&g->dX, sizeof(double) * M * D));
  GK(cudaMalloc(&g->dL, sizeof(double) * (size_t)Mp * Mp));
  GK(cudaMalloc(&g->dalpha, sizeof(double) * Mp));
  GK(cudaMalloc(&g->dwork, sizeof(double) * 2 * Mp));
  GK(cudaMalloc(&dy, sizeof(double) * M));
  GK(cudaMalloc(&dstatus, sizeof(int)));
  GK(cudaMemcpyAsync(g->dX, X, sizeof(double) * M * D, cudaMemcpyHostToDevice, s));
  if (y) GK(cudaMemcpyAsync(dy, y, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  GK(cudaMemsetAsync(dstatus, 0, sizeof(int), s));
  if (mu_X) {
    GK(cudaMalloc(&dmuX, sizeof(double) * M));
    GK(cudaMemcpyAsync(dmuX, mu_X, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  }
  if (fixed) {
    GK(cudaMalloc(&dfixed, sizeof(double) * D));
    GK(cudaMemcpyAsync(dfixed, fixed, sizeof(double) * D, cudaMemcpyHostToDevice, s));
  }
  const Fallback fallback = make_fallback(p, D);
  // the pair-separation row sums (M x D) use the factor's storage before
  // the covariance fills it
  if (!fixed) {
    k_gp_pairsep<<<M, 128, 0, s>>>(g->dX, M, D, g->dL);
    g->launches++;
  }
  k_gp_scales<<<1, 256, 0, s>>>(g->dL, g->dscale, M, D, fallback, dfixed);
  k_gp_cov<<<dim3((Mp + 127) / 128, Mp), 128, 0, s>>>(g->dX, M, Mp, D, g->dscale, g->sf2, g->l2, g->sn2, g->dL);
  g->launches += 2;
  const int nt = Mp / TB;
  if (nt >= kLookaheadTiles && g->fs[0]) {
    const int st = enqueue_cholesky_lookahead(g, dstatus);
    if (st) return st;
  } else {
    for (int kb = 0; kb < nt; ++kb) {
      k_potrf_diag<<<1, 4 * TB, 0, s>>>(g->dL, Mp, kb, dstatus);
      g->launches++;
      const int rest = nt - kb - 1;
      if (rest > 0) {
        k_trsm_panel<<<rest * (TB / kTrsmRows), dim3(TB, kTrsmRows), 0, s>>>(g->dL, Mp, kb);
        k_syrk_update<<<rest * (rest + 1) / 2, dim3(TB, TB), 0, s>>>(g->dL, Mp, kb, nt, 0);
        g->launches += 2;
      }
    }
  }
  if (g->has_alpha) {
    const int st = enqueue_alpha(g, dy, dmuX);
    if (st) return st;
  }
  int status = 0;
  GK(cudaGetLastError());
  GK(cudaMemcpyAsync(&status, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
  GK(cudaStreamSynchronize(s));
  return status ? status : MDGP_OK;
}

extern "C" {

static int gp_fit_entry(mdgp_ctx* ctx, const double* X, const double* y, int64_t M, int32_t D,
                        const mdgp_gp_params* params, const double* mu_X, bool with_alpha, mdgp_gp** out) {
  if (!ctx || !params || !out || M < 0 || M > kMaxM || D < 1 || D > kMaxD) return MDGP_E_ARG;
  if (M > 0 && (!X || (with_alpha && !y))) return MDGP_E_ARG;
  if (!(params->sf2 > 0) || !(params->l2 > 0) || !(params->sn2 >= 0)) return MDGP_E_ARG;
  if (!(params->period >= 0) || (params->period > 0 && (D != 1 || params->fixed_scales))) return MDGP_E_ARG;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  mdgp_gp* g = new (std::nothrow) mdgp_gp();
  if (!g) return MDGP_E_NOMEM;
  g->device = ctx->device;
  g->stream = ctx->stream;
  g->M = (int)M;
  g->Mp = (int)((M + TB - 1) / TB * TB);
  g->D = D;
  g->sf2 = params->sf2;
  g->l2 = params->l2;
  g->sn2 = params->sn2;
  g->period = params->period;
  g->has_alpha = with_alpha;
  for (int k = 0; k < 2; ++k) g->fs[k] = ctx->fact_stream[k];
  for (int k = 0; k < 4; ++k) g->fe[k] = ctx->fact_event[k];
  int st = gp_fit_impl(g, X, with_alpha ? y : nullptr, with_alpha ? mu_X : nullptr, params);
  if (st != MDGP_OK) {
    std::snprintf(ctx->err, sizeof(ctx->err), "gp fit: %s", g->err[0] ? g->err : "not positive definite");
    gp_release(g);
    delete g;
    return st;
  }
  *out = g;
  return MDGP_OK;
}

int mdgp_gp_fit(mdgp_ctx* ctx, const double* X, const double* y, int64_t M, int32_t D,
                const mdgp_gp_params* params, const double* mu_X, mdgp_gp** out) {
  return gp_fit_entry(ctx, X, y, M, D, params, mu_X, true, out);
}

int mdgp_gp_predict(mdgp_gp* g, const double* Xs, int64_t m, const double* mu_Xs, double* mean, double* var) {
  if (!g || m < 0 || (m > 0 && (!Xs || (!mean && !var)))) return MDGP_E_ARG;
  if (m == 0) return MDGP_OK;
  cudaSetDevice(g->device);
  if (g->M == 0) {  // empty database: the prior (paper Sec. 3.1)
    for (int64_t q = 0; q < m; ++q) {
      if (mean) mean[q] = mu_Xs ? mu_Xs[q] : 0.0;
      if (var) var[q] = g->sf2;
    }
    return MDGP_OK;
  }
  cudaStream_t s = g->stream;
  if ((size_t)m > g->qcap) {
    for (double** p : {&g->dq, &g->dmu, &g->dmean, &g->dvar})
      if (*p) { cudaFree(*p); *p = nullptr; }
    GK(cudaMalloc(&g->dq, sizeof(double) * m * g->D));
    GK(cudaMalloc(&g->dmu, sizeof(double) * m));
    GK(cudaMalloc(&g->dmean, sizeof(double) * m));
    GK(cudaMalloc(&g->dvar, sizeof(double) * m));
    g->qcap = (size_t)m;
  }
  GK(cudaMemcpyAsync(g->dq, Xs, sizeof(double) * m * g->D, cudaMemcpyHostToDevice, s));
  if (mu_Xs) GK(cudaMemcpyAsync(g->dmu, mu_Xs, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  const size_t smem = sizeof(double) * g->Mp;
  GK(allow_solve_smem());
  k_gp_predict<<<(unsigned)m, 256, smem, s>>>(g->dX, g->dL, g->has_alpha ? g->dalpha : nullptr, g->dscale, g->M,
                                              g->Mp, g->D, g->sf2, g->l2, g->dq, mu_Xs ? g->dmu : nullptr,
                                              g->dmean, g->dvar, var != nullptr);
  g->launches++;
  GK(cudaGetLastError());
  if (mean) GK(cudaMemcpyAsync(mean, g->dmean, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  if (var) GK(cudaMemcpyAsync(var, g->dvar, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  GK(cudaStreamSynchronize(s));
  return MDGP_OK;
}

int mdgp_gp_set_outputs(mdgp_gp* g, const double* y, const double* mu_X) {
  if (!g || (g->M > 0 && !y)) return MDGP_E_ARG;
  if (g->M == 0) {
    g->has_alpha = true;
    return MDGP_OK;
  }
  cudaSetDevice(g->device);
  cudaStream_t s = g->stream;
  const int M = g->M;
  double *dy = nullptr, *dmu = nullptr;
  cudaError_t e = cudaMalloc(&dy, sizeof(double) * M);
  if (e == cudaSuccess && mu_X) e = cudaMalloc(&dmu, sizeof(double) * M);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, sizeof(double) * M, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && mu_X) e = cudaMemcpyAsync(dmu, mu_X, sizeof(double) * M, cudaMemcpyHostToDevice, s);
  int st = e == cudaSuccess ? MDGP_OK : gp_err(g, e);
  if (st == MDGP_OK) st = enqueue_alpha(g, dy, dmu);
  if (st == MDGP_OK) {
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = gp_err(g, e);
  }
  if (dy) cudaFree(dy);
  if (dmu) cudaFree(dmu);
  if (st == MDGP_OK) g->has_alpha = true;
  return st;
}

int mdgp_gp_log_marginal(const mdgp_gp* g, double* lml) {
  if (!g || !lml || !g->has_alpha) return MDGP_E_ARG;
  if (g->M == 0) { *lml = 0.0; return MDGP_OK; }
  cudaSetDevice(g->device);
  double t[2];
  if (cudaMemcpy(t, g->dscale + kMaxD, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess) return MDGP_E_CUDA;
  *lml = -0.5 * t[0] - t[1] - 0.5 * g->M * std::log(2.0 * M_PI);
  return MDGP_OK;
}

// Evidence of one hyperparameter set: a fit, its log marginal likelihood;
// a covariance that is not positive definite scores -inf.
static int evidence(mdgp_ctx* ctx, const double* X, const double* y, int64_t M, int32_t D,
                    const mdgp_gp_params& p, const double* mu_X, double* lml) {
  mdgp_gp* g = nullptr;
  const int st = mdgp_gp_fit(ctx, X, y, M, D, &p, mu_X, &g);
  if (st == MDGP_E_NOTPD) { *lml = -INFINITY; return MDGP_OK; }
  if (st) return st;
  const int st2 = mdgp_gp_log_marginal(g, lml);
  mdgp_gp_free(g);
  return st2;
}

int mdgp_gp_optimize(mdgp_ctx* ctx, const double* X, const double* y, int64_t M, int32_t D,
                     const mdgp_gp_params* start, const double* mu_X, int32_t max_evals, mdgp_gp_params* best,
                     double* best_lml) {
  if (!ctx || !start || !best || M < 1 || max_evals < 1) return MDGP_E_ARG;
  mdgp_gp_params cur = *start;
  double f = 0.0;
  int st = evidence(ctx, X, y, M, D, cur, mu_X, &f);
  if (st) return st;
  int evals = 1;
  double step = 4.0;   // multiplicative step in each hyperparameter
  while (step > 1.05 && evals < max_evals) {
    bool moved = false;
    for (int k = 0; k < 3 && evals < max_evals; ++k) {
      if (start->hold & (1 << k)) continue;
      double* v = k == 0 ? &cur.sf2 : (k == 1 ? &cur.l2 : &cur.sn2);
      const double v0 = *v;
      double bestv = v0, bestf = f;
      for (int dir = 0; dir < 2 && evals < max_evals; ++dir) {
        *v = dir == 0 ? v0 * step : v0 / step;
        double ft = 0.0;
        if ((st = evidence(ctx, X, y, M, D, cur, mu_X, &ft))) { *best = *start; return st; }
        ++evals;
        // a move must gain more than rounding can explain
        if (ft > bestf + 1e-9 * std::fabs(bestf) + 1e-12) { bestf = ft; bestv = *v; }
      }
      *v = bestv;
      if (bestv != v0) { f = bestf; moved = true; }
    }
    if (!moved) step = std::sqrt(step);
  }
  *best = cur;
  if (best_lml) *best_lml = f;
  return MDGP_OK;
}

int mdgp_gp_scales(const mdgp_gp* g, double* scales) {
  if (!g || !scales) return MDGP_E_ARG;
  cudaSetDevice(g->device);
  if (cudaMemcpy(scales, g->dscale, sizeof(double) * g->D, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MDGP_E_CUDA;
  if (g->period > 0.0) scales[0] = g->period;   // the periodic kernel: its period
  return MDGP_OK;
}

int mdgp_gp_free(mdgp_gp* g) {
  if (!g) return MDGP_E_ARG;
  cudaSetDevice(g->device);
  gp_release(g);
  delete g;
  return MDGP_OK;
}

int mdgp_gp_fit_inputs(mdgp_ctx* ctx, const double* X, int64_t M, int32_t D, const mdgp_gp_params* params,
                       mdgp_gp** out) {
  return gp_fit_entry(ctx, X, nullptr, M, D, params, nullptr, false, out);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free GP posterior.
//
// For callers that cannot call cudaMalloc while they run: an application
// whose device memory is all handed to its own pool allocator up front, or a
// latency-bound control loop where an allocation (which may synchronise the
// device) is not acceptable.  The factorisation lives in one file-scope
// device array of a fixed size instead of in buffers from cudaMalloc.  Every
// GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxM = 512;   // largest database this entry point accepts
constexpr size_t kNoAllocL = (size_t)kNoAllocMaxM * kNoAllocMaxM;
// layout: Cholesky factor [512 x 512] | alpha [512] | scales [8] | status word
constexpr size_t kNoAllocDoubles = kNoAllocL + kNoAllocMaxM + kMaxD + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kNoAllocMaxDevices = 64;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the symbol name is only a host-side handle).
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return MDGP_E_ARG;
  if (!g_noalloc_ptr[device]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) return MDGP_E_CUDA;
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return MDGP_OK;
}

}  // namespace

extern "C" int mdgp_gp_posterior_noalloc(const double* X, const double* y, int64_t M, int32_t D,
                                         const mdgp_gp_params* params, const double* mu_X, const double* Xs,
                                         int64_t m, const double* mu_Xs, double* mean, double* var,
                                         void* stream) {
  if (!params || M < 1 || D < 1 || D > kMaxD || m < 0 || !X || !y || (m > 0 && (!Xs || !mean || !var)))
    return MDGP_E_ARG;
  if (M > kNoAllocMaxM) return MDGP_E_LIMIT;  // the scratch array holds at most 512 entries
  if (!(params->sf2 > 0) || !(params->l2 > 0) || !(params->sn2 >= 0) || params->fixed_scales || params->period != 0.0)
    return MDGP_E_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MDGP_E_CUDA;
  double* base = nullptr;
  int st = noalloc_scratch(device, &base);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (allow_solve_smem() != cudaSuccess) return MDGP_E_CUDA;
  const int Mi = (int)M, Mp = (int)((M + TB - 1) / TB * TB);
  double* L = base;
  double* alpha = base + kNoAllocL;
  double* scale = alpha + kNoAllocMaxM;
  int* status = (int*)(scale + kMaxD);
  // the scratch keeps the previous call's contents: clear the accumulators
  if (cudaMemsetAsync(scale, 0, sizeof(double) * (kMaxD + 8), s) != cudaSuccess) return MDGP_E_CUDA;
  const Fallback fallback = make_fallback(params, D);
  k_gp_pairsep<<<Mi, 128, 0, s>>>(X, Mi, D, L);   // row sums in the factor's space, before the covariance
  k_gp_scales<<<1, 256, 0, s>>>(L, scale, Mi, D, fallback, nullptr);
  // the factor is laid out with leading dimension Mp inside the fixed array
  k_gp_cov<<<dim3((Mp + 127) / 128, Mp), 128, 0, s>>>(X, Mi, Mp, D, scale, params->sf2, params->l2, params->sn2,
                                                      L);
  const int nt = Mp / TB;
  for (int kb = 0; kb < nt; ++kb) {
    k_potrf_diag<<<1, 4 * TB, 0, s>>>(L, Mp, kb, status);
    const int rest = nt - kb - 1;
    if (rest > 0) {
      k_trsm_panel<<<rest * (TB / kTrsmRows), dim3(TB, kTrsmRows), 0, s>>>(L, Mp, kb);
      k_syrk_update<<<rest * (rest + 1) / 2, dim3(TB, TB), 0, s>>>(L, Mp, kb, nt, 0);
    }
  }
  k_gp_alpha<<<1, 256, sizeof(double) * Mp, s>>>(L, Mi, Mp, y, mu_X, alpha, nullptr);
  if (m > 0)
    k_gp_predict<<<(unsigned)m, 256, sizeof(double) * Mp, s>>>(X, L, alpha, scale, Mi, Mp, D, params->sf2,
                                                               params->l2, Xs, mu_Xs, mean, var, true);
  if (cudaGetLastError() != cudaSuccess) return MDGP_E_CUDA;
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MDGP_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MDGP_E_CUDA;
  return h_status ? h_status : MDGP_OK;
}
