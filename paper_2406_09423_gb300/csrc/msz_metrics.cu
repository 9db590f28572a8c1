// Evaluation metrics of an edited field against the original (Appendix B:
// PSNR and the right labelled ratio). No counterpart in the correction
// loop: it measures what the loop preserves (the labels) and what it costs
// (the distortion).
//
// Labels are those of Sec. 3: a vertex's maximum / minimum label is the
// extremum its steepest ascending / descending line reaches. Here they come
// from dense pointer doubling over the whole field (P <- P o P until no
// pointer changes), for f and g at once; the correction loop's own labelling
// (tiles + exit table) is not used, so the two paths check each other.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "msz.h"
#include "msz_device.cuh"

namespace msz {
namespace {

constexpr int kMetricThreads = 256;

bool metric_geom(int ndim, const int64_t* dims, Geom& G) {
  if ((ndim != 2 && ndim != 3) || !dims) return false;
  const int64_t nx = dims[0], ny = dims[1], nz = (ndim == 3) ? dims[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1) return false;
  const int64_t n = nx * ny * nz;
  if (nx > 0x7fffffff || ny > 0x7fffffff || nz > 0x7fffffff || n > 0x7fffffffLL) return false;
  G.nx = (int)nx;
  G.ny = (int)ny;
  G.nz = (int)nz;
  G.nxny = (int)(nx * ny);
  G.n = (int)n;
  G.nd = ndim;
  G.dx = fast_div((uint32_t)nx);
  G.dy = fast_div((uint32_t)ny);
  return true;
}

// Block sums / minima / maxima of double values, written per block (the host
// combines them in block order, so the result does not depend on timing).
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t += s[w];
  return t;
}

// Pointers of f and g (ascending, descending: the steepest vertex of the
// closed 1-ring), and per block: the sum of (f - g)^2 in double, min f, max f.
template <class T, int ND>
__global__ void __launch_bounds__(kMetricThreads)
    k_metric_init(const T* __restrict__ f, const T* __restrict__ g, Geom G, int32_t* pfu, int32_t* pfd, int32_t* pgu,
                  int32_t* pgd, double* part) {
  __shared__ double s[kMetricThreads / 32];
  double sq = 0.0, lo = INFINITY, hi = -INFINITY;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(G, v, x, y, z);
    const uint8_t df = direction_of<T, ND>(f, G, v, x, y, z);
    const uint8_t dg = direction_of<T, ND>(g, G, v, x, y, z);
    pfu[v] = v + slot_offset(df & 15, ND, G.nx, G.nxny);
    pfd[v] = v + slot_offset(df >> 4, ND, G.nx, G.nxny);
    pgu[v] = v + slot_offset(dg & 15, ND, G.nx, G.nxny);
    pgd[v] = v + slot_offset(dg >> 4, ND, G.nx, G.nxny);
    const double fv = (double)f[v], d = fv - (double)g[v];
    sq += d * d;
    lo = fmin(lo, fv);
    hi = fmax(hi, fv);
  }
  const double ssum = block_sum<kMetricThreads>(sq, s);
  // minimum and maximum through the same reduction shape
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(kFull, lo, o));
    hi = fmax(hi, __shfl_xor_sync(kFull, hi, o));
  }
  __shared__ double slo[kMetricThreads / 32], shi[kMetricThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < kMetricThreads / 32; ++w) {
      lo = fmin(lo, slo[w]);
      hi = fmax(hi, shi[w]);
    }
    part[3 * blockIdx.x + 0] = ssum;
    part[3 * blockIdx.x + 1] = lo;
    part[3 * blockIdx.x + 2] = hi;
  }
}

// One doubling round on the four pointer arrays; *changed is set when a
// pointer moved.
__global__ void __launch_bounds__(kMetricThreads)
    k_metric_jump(int n, int32_t* p0, int32_t* p1, int32_t* p2, int32_t* p3, int* changed) {
  int moved = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t* P[4] = {p0, p1, p2, p3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int32_t a = P[k][v], b = P[k][a];
      if (b != a) {
        P[k][v] = b;
        moved = 1;
      }
    }
  }
  if (__syncthreads_or(moved) && threadIdx.x == 0) atomicExch(changed, 1);
}

// Vertices whose maximum or minimum label differs between f and g, per block.
__global__ void __launch_bounds__(kMetricThreads)
    k_metric_wrong(int n, const int32_t* pfu, const int32_t* pfd, const int32_t* pgu, const int32_t* pgd,
                   unsigned long long* wrong) {
  unsigned long long w = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    w += (pfu[v] != pgu[v] || pfd[v] != pgd[v]) ? 1ull : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(wrong, w);
}

}  // namespace
}  // namespace msz

using namespace msz;

int msz_field_metrics(const void* f_dev, const void* g_dev, int ndim, const int64_t dims[3], int dtype, void* stream,
                      msz_metric_values* out) {
  Geom G;
  if (!metric_geom(ndim, dims, G)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  if (!f_dev || !g_dev || !out) return MSZ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MSZ_ERR_CUDA;
  const size_t n = (size_t)G.n;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + kMetricThreads - 1) / kMetricThreads, (size_t)sms * 8));
  // scratch: four pointer arrays, the block partials, the flag and the count
  const size_t ptr_bytes = 4 * n * sizeof(int32_t), part_bytes = 3 * (size_t)blocks * sizeof(double);
  unsigned char* scratch = nullptr;
  if (cudaMallocAsync(&scratch, ptr_bytes + part_bytes + 16, s) != cudaSuccess) {
    cudaGetLastError();
    return MSZ_ERR_OOM;
  }
  int32_t* pfu = reinterpret_cast<int32_t*>(scratch);
  int32_t* pfd = pfu + n;
  int32_t* pgu = pfd + n;
  int32_t* pgd = pgu + n;
  double* part = reinterpret_cast<double*>(scratch + ptr_bytes);
  int* changed = reinterpret_cast<int*>(scratch + ptr_bytes + part_bytes);
  unsigned long long* wrong = reinterpret_cast<unsigned long long*>(scratch + ptr_bytes + part_bytes + 8);
  int status = MSZ_OK;
  auto fail = [&](int st) {
    if (status == MSZ_OK) status = st;
  };
  if (dtype == MSZ_F32) {
    const float* f = static_cast<const float*>(f_dev);
    const float* g = static_cast<const float*>(g_dev);
    if (ndim == 3) k_metric_init<float, 3><<<blocks, kMetricThreads, 0, s>>>(f, g, G, pfu, pfd, pgu, pgd, part);
    else k_metric_init<float, 2><<<blocks, kMetricThreads, 0, s>>>(f, g, G, pfu, pfd, pgu, pgd, part);
  } else {
    const double* f = static_cast<const double*>(f_dev);
    const double* g = static_cast<const double*>(g_dev);
    if (ndim == 3) k_metric_init<double, 3><<<blocks, kMetricThreads, 0, s>>>(f, g, G, pfu, pfd, pgu, pgd, part);
    else k_metric_init<double, 2><<<blocks, kMetricThreads, 0, s>>>(f, g, G, pfu, pfd, pgu, pgd, part);
  }
  // pointer doubling to the labels: lines are acyclic, so fewer than 32
  // rounds reach the fixed point of a field of at most 2^31 vertices
  bool fixed = false;
  for (int r = 0; r < 64 && status == MSZ_OK; ++r) {
    int h = 0;
    if (cudaMemsetAsync(changed, 0, sizeof(int), s) != cudaSuccess) fail(MSZ_ERR_CUDA);
    k_metric_jump<<<blocks, kMetricThreads, 0, s>>>(G.n, pfu, pfd, pgu, pgd, changed);
    if (cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      fail(MSZ_ERR_CUDA);
    if (!h) {
      fixed = true;
      break;
    }
  }
  if (status == MSZ_OK && !fixed) fail(MSZ_ERR_TIMEOUT);
  std::vector<double> hp(3 * (size_t)blocks);
  unsigned long long hw = 0;
  if (status == MSZ_OK) {
    if (cudaMemsetAsync(wrong, 0, sizeof(unsigned long long), s) != cudaSuccess) fail(MSZ_ERR_CUDA);
    k_metric_wrong<<<blocks, kMetricThreads, 0, s>>>(G.n, pfu, pfd, pgu, pgd, wrong);
    if (cudaMemcpyAsync(hp.data(), part, part_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hw, wrong, sizeof(hw), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      fail(MSZ_ERR_CUDA);
  }
  cudaFreeAsync(scratch, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) fail(MSZ_ERR_CUDA);
  if (status != MSZ_OK) return status;
  double sum = 0.0, lo = INFINITY, hi = -INFINITY;
  for (int b = 0; b < blocks; ++b) {
    sum += hp[3 * b];
    lo = std::min(lo, hp[3 * b + 1]);
    hi = std::max(hi, hp[3 * b + 2]);
  }
  out->mse = sum / (double)n;
  out->value_range = hi - lo;
  out->psnr = out->mse == 0.0 ? INFINITY : 20.0 * std::log10(out->value_range / std::sqrt(out->mse));
  out->wrong = hw;
  out->right_labelled = 1.0 - (double)hw / (double)n;
  return MSZ_OK;
}
