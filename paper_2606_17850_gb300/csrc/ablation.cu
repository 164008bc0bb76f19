// CSR sparse matrix-vector product of the same system, for the stencil-vs-CSR
// comparison of Sec. 5.5 (Ablation Study I, Table abl_spmv: the paper measures its
// diagonal-wise SpMV against a CSR baseline with row-wise SpMV on the same
// matrices).  Not on the solve path.
//
// The matrix is assembled on the device from the FP64 face conductances in
// compressed sparse row form: row i lists its existing neighbours in ascending
// column order (z-1, y-1, x-1, diagonal, x+1, y+1, z+1) with values -g and the
// diagonal s_z + sum g.  Row offsets follow in closed form from the geometry (a
// row has 1 + one entry per existing neighbour), so no scan is needed.
//
// Two products: one thread per row (scalar CSR, the paper's row-wise baseline)
// and eight lanes per row with a shuffle reduction (vector CSR).
#include <algorithm>

#include "internal.h"

namespace {

// sum over x' < x of ([x' > 0] + [x' < n-1]): neighbour entries of the first x
// cells of a line of n cells
__device__ __forceinline__ long long nb_prefix(long long n, long long x) {
  return (x > 1 ? x - 1 : 0) + (x < n - 1 ? x : n - 1);
}

__device__ __forceinline__ long long row_start(const Dims& d, int x, int y, int z) {
  const long long nx = d.nx, ny = d.ny, L = d.L, pxy = d.pxy;
  const long long X = nb_prefix(nx, nx), Y = nb_prefix(ny, ny);
  const long long ey = (y > 0) + (y < ny - 1), ez = (z > 0) + (z < L - 1);
  long long s = (long long)z * (pxy + ny * X + nx * Y) + pxy * nb_prefix(L, z);      // whole layers below
  s += (long long)y * (nx + X) + nx * nb_prefix(ny, y) + (long long)y * nx * ez;      // whole rows below
  s += (long long)x + nb_prefix(nx, x) + (long long)x * (ey + ez);                    // cells to the left
  return s;
}

template <typename TV>
__global__ void k_build_csr(Dims d, Faces64 f, const LayerTab* tab, int* __restrict__ rp, int* __restrict__ col,
                            TV* __restrict__ val) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const long long i = c.i, nx = d.nx, pxy = d.pxy;
  long long k = row_start(d, c.x, c.y, c.z);
  rp[i] = (int)k;
  if (i == d.n - 1) rp[d.n] = (int)row_start(d, c.x, c.y, c.z) + 1 + (c.x > 0) + (c.y > 0) + (c.z > 0);
  double diag = tab->s64[c.z];
  auto put = [&](long long j, double g) {
    col[k] = (int)j;
    val[k] = (TV)(-g);
    ++k;
    diag += g;
  };
  if (c.z > 0) put(i - pxy, f.gz[i - pxy]);
  if (c.y > 0) put(i - nx, f.gy[i - nx]);
  if (c.x > 0) put(i - 1, f.gx[i - 1]);
  const long long kd = k++;
  if (c.x + 1 < d.nx) put(i + 1, f.gx[i]);
  if (c.y + 1 < d.ny) put(i + nx, f.gy[i]);
  if (c.z + 1 < d.L) put(i + pxy, f.gz[i]);
  col[kd] = (int)i;
  val[kd] = (TV)diag;
}

template <typename TV>
__global__ void __launch_bounds__(256) k_csr_scalar(long long n, const int* __restrict__ rp, const int* __restrict__ col,
                                                    const TV* __restrict__ val, const TV* __restrict__ x,
                                                    TV* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TV acc = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) acc += val[k] * x[col[k]];
  y[i] = acc;
}

template <typename TV>
__global__ void __launch_bounds__(256) k_csr_vector(long long n, const int* __restrict__ rp, const int* __restrict__ col,
                                                    const TV* __restrict__ val, const TV* __restrict__ x,
                                                    TV* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long i = t >> 3;
  const int lane = (int)(t & 7);
  TV acc = 0;
  if (i < n) {
    const int k = rp[i] + lane;
    if (k < rp[i + 1]) acc = val[k] * x[col[k]];
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, 8);
  if (i < n && lane == 0) y[i] = acc;
}

struct CsrMat {
  int *rp = nullptr, *col = nullptr;
  void* val = nullptr;
  ~CsrMat() {
    cudaFree(rp);
    cudaFree(col);
    cudaFree(val);
  }
};

}  // namespace

extern "C" th_status thermal_csr_spmv(thermal_grid* g, int variant, int precision, double dt, const void* x, void* y,
                                      int reps, double* ms, void* stream) {
  try {
    th_clear_error();
    if (!g || !x || !y) return th_fail(TH_EINVAL, "NULL argument");
    if (x == y) return th_fail(TH_EINVAL, "x and y must not alias");
    if (variant != 0 && variant != 1) return th_fail(TH_EINVAL, "variant must be 0 (scalar) or 1 (vector)");
    if (precision != TH_PREC_FP64 && precision != TH_PREC_MIXED_IR)
      return th_fail(TH_EINVAL, "precision must be TH_PREC_FP64 or TH_PREC_MIXED_IR (FP32)");
    if (reps < 1) return th_fail(TH_EINVAL, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    TH_TRY(grid_ensure_tab(g, dt, s));
    const Dims d = grid_dims(g);
    const long long n = g->n;
    const long long nnz = n + 2LL * ((long long)(g->nx - 1) * g->ny * g->L + (long long)g->nx * (g->ny - 1) * g->L +
                                     (long long)g->nx * g->ny * (g->L - 1));
    if (nnz >= (1LL << 31)) return th_fail(TH_EINVAL, "CSR with %lld entries exceeds 32-bit offsets", nnz);
    const bool f64 = precision == TH_PREC_FP64;
    const size_t vs = f64 ? sizeof(double) : sizeof(float);
    CsrMat m;
    TH_CUDA(cudaMalloc(&m.rp, sizeof(int) * (size_t)(n + 1)));
    TH_CUDA(cudaMalloc(&m.col, sizeof(int) * (size_t)nnz));
    TH_CUDA(cudaMalloc(&m.val, vs * (size_t)nnz));
    const dim3 gb = grid_blocks(g), tb(TH_BX, TH_BY);
    if (f64)
      k_build_csr<double><<<gb, tb, 0, s>>>(d, g->f64, g->tab, m.rp, m.col, (double*)m.val);
    else
      k_build_csr<float><<<gb, tb, 0, s>>>(d, g->f64, g->tab, m.rp, m.col, (float*)m.val);
    TH_CHECK_LAUNCH();
    const unsigned nb = (unsigned)(((variant == 0 ? n : 8 * n) + 255) / 256);
    auto launch = [&]() {
      if (f64) {
        if (variant == 0)
          k_csr_scalar<double><<<nb, 256, 0, s>>>(n, m.rp, m.col, (const double*)m.val, (const double*)x, (double*)y);
        else
          k_csr_vector<double><<<nb, 256, 0, s>>>(n, m.rp, m.col, (const double*)m.val, (const double*)x, (double*)y);
      } else {
        if (variant == 0)
          k_csr_scalar<float><<<nb, 256, 0, s>>>(n, m.rp, m.col, (const float*)m.val, (const float*)x, (float*)y);
        else
          k_csr_vector<float><<<nb, 256, 0, s>>>(n, m.rp, m.col, (const float*)m.val, (const float*)x, (float*)y);
      }
    };
    launch();  // warm-up (and the result when reps == 1)
    TH_CHECK_LAUNCH();
    if (ms) {
      cudaEvent_t a, b;
      TH_CUDA(cudaEventCreate(&a));
      TH_CUDA(cudaEventCreate(&b));
      cudaEventRecord(a, s);
      for (int r = 0; r < reps; ++r) launch();
      cudaEventRecord(b, s);
      const cudaError_t e = cudaEventSynchronize(b);
      float t = 0.f;
      cudaEventElapsedTime(&t, a, b);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      if (e != cudaSuccess) return th_fail(TH_ECUDA, "CSR timing failed: %s", cudaGetErrorString(e));
      *ms = (double)t / reps;
    }
    TH_CHECK_LAUNCH();
    // the matrix is freed when m goes out of scope: finish the stream's use of it first
    TH_CUDA(cudaStreamSynchronize(s));
    return TH_OK;
  } catch (const std::bad_alloc&) {
    return th_fail(TH_ENOMEM, "host allocation failed");
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}
