// Uniform 2^d tree on the GPU (Sec. 2.1): bounding hypercube, leaf cell and
// Morton key per point, stable counting sort into tree order, per-level box
// ranges.  All integer decisions are bit-identical to the definition:
// cell_k = min(floor(((p_k - lo_k) * n) / side), n - 1), n = 2^L.
#include "internal.h"

namespace aifmm {

namespace {

// AoS (N x d, row-major) -> SoA [d][N]
__global__ void k_aos_to_soa(const double* __restrict__ aos, int N, int d, double* __restrict__ soa) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    for (int k = 0; k < d; ++k) soa[(size_t)k * N + i] = aos[(size_t)i * d + k];
}

// bounding hypercube: lo_k = min_k, side = max_k (max_k - lo_k); one block
__global__ void k_bbox(const double* __restrict__ soa, int N, int d, double* __restrict__ out) {
  __shared__ double smin[3][32], smax[3][32];
  double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    for (int k = 0; k < d; ++k) {
      double v = soa[(size_t)k * N + i];
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < d; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if (lane == 0) {
      smin[k][w] = lo[k];
      smax[k][w] = hi[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    double side = 0.0;
    for (int k = 0; k < d; ++k) {
      double a = smin[k][0], b = smax[k][0];
      for (int q = 1; q < nw; ++q) {
        a = fmin(a, smin[k][q]);
        b = fmax(b, smax[k][q]);
      }
      out[k] = a;
      side = fmax(side, b - a);
    }
    out[3] = side;
  }
}

__global__ void k_leaf_keys(const double* __restrict__ soa, int N, int d, int L,
                            const double* __restrict__ bbox, int* __restrict__ key,
                            int* __restrict__ count) {
  const double n = (double)(1 << L);
  const double side = bbox[3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
      double t = __ddiv_rn(__dmul_rn(__dsub_rn(soa[(size_t)k * N + i], bbox[k]), n), side);
      int ci = (int)floor(t);
      c[k] = ci < (1 << L) - 1 ? ci : (1 << L) - 1;
    }
    int kk = morton_key(c, d, L);
    key[i] = kk;
    atomicAdd(&count[kk], 1);
  }
}

// exclusive scan of count[0..n) into start[0..n]; single block
__global__ void k_scan(const int* __restrict__ count, int n, int* __restrict__ start) {
  __shared__ int carry;
  __shared__ int buf[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < n ? count[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) start[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_scatter(const int* __restrict__ key, int N, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int k = key[i];
    int pos = start[k] + atomicAdd(&fill[k], 1);
    out[pos] = i;
  }
}

// sort each leaf segment by original index (stable tree order); one block per
// leaf, rank sort in shared memory; segments longer than cap raise CAPACITY.
__global__ void k_sort_segments(const int* __restrict__ start, const int* __restrict__ in,
                                int* __restrict__ out, int cap, int* err) {
  extern __shared__ int seg[];
  int b = blockIdx.x;
  int s = start[b], e = start[b + 1], n = e - s;
  if (n > cap) {
    set_err(err, DERR_CAPACITY);
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) seg[i] = in[s + i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int v = seg[i], rnk = 0;
    for (int j = 0; j < n; ++j) rnk += seg[j] < v;
    out[s + rnk] = v;
  }
}

__global__ void k_gather_points(const double* __restrict__ soa_in, const int* __restrict__ perm,
                                int N, int d, double* __restrict__ soa_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int p = perm[i];
    for (int k = 0; k < d; ++k) soa_out[(size_t)k * N + i] = soa_in[(size_t)k * N + p];
  }
}

// duplicate points make log and 1/r kernels singular: flag them.  Points in
// tree order; equal points fall into the same leaf, so a check inside each
// leaf segment is complete.
__global__ void k_check_duplicates(const double* __restrict__ soa, int N, int d,
                                   const int* __restrict__ start, int* err) {
  int b = blockIdx.x;
  int s = start[b], e = start[b + 1];
  for (int i = s + threadIdx.x; i < e; i += blockDim.x)
    for (int j = s; j < i; ++j) {
      bool same = true;
      for (int k = 0; k < d; ++k) same = same && soa[(size_t)k * N + i] == soa[(size_t)k * N + j];
      if (same) set_err(err, DERR_DUPLICATE);
    }
}

__global__ void k_level_starts(const int* __restrict__ leaf_start, int shift, int nb, int* __restrict__ out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x)
    out[b] = leaf_start[(size_t)b << shift];
}

}  // namespace

int build_tree(Handle& h, const double* aos) {
  const int N = (int)h.N, d = h.d, L = h.L;
  cudaStream_t st = h.stream;
  const int nleaf = 1 << (d * L);
  double* soa = hnew<double>(h, (size_t)d * N, false);
  double* soa2 = hnew<double>(h, (size_t)d * N, false);
  int* key = hnew<int>(h, N, false);
  int* count = hnew<int>(h, nleaf);
  int* fill = hnew<int>(h, nleaf);
  int* tmp = hnew<int>(h, N, false);
  h.perm = hnew<int>(h, N, false);
  h.bbox = hnew<double>(h, 4);
  // level starts for all levels, concatenated
  h.soff.assign(L + 2, 0);
  for (int l = 0; l <= L; ++l) h.soff[l + 1] = h.soff[l] + (1 << (d * l)) + 1;
  h.start = hnew<int>(h, h.soff[L + 1]);
  if (!soa || !soa2 || !key || !count || !fill || !tmp || !h.perm || !h.bbox || !h.start) return HOOM;
  int grid = (N + 255) / 256;
  if (grid > 4096) grid = 4096;
  k_aos_to_soa<<<grid, 256, 0, st>>>(aos, N, d, soa); ++h.nlaunch;
  k_bbox<<<1, 1024, 0, st>>>(soa, N, d, h.bbox); ++h.nlaunch;
  k_leaf_keys<<<grid, 256, 0, st>>>(soa, N, d, L, h.bbox, key, count); ++h.nlaunch;
  int* leaf_start = h.start + h.soff[L];
  k_scan<<<1, 1024, 0, st>>>(count, nleaf, leaf_start); ++h.nlaunch;
  k_scatter<<<grid, 256, 0, st>>>(key, N, leaf_start, fill, tmp); ++h.nlaunch;
  // leaf occupancy bound for the shared-memory rank sort
  h.h_leaf_start.resize(nleaf + 1);
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(h.h_leaf_start.data(), leaf_start, sizeof(int) * (nleaf + 1),
                                    cudaMemcpyDeviceToHost, st));
  AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
  int occ = 0;
  for (int b = 0; b < nleaf; ++b) occ = std::max(occ, h.h_leaf_start[b + 1] - h.h_leaf_start[b]);
  const int cap = 12 * 1024;  // 48 KB of shared memory
  if (occ > cap) {
    h.err = "leaf box holds " + std::to_string(occ) + " points; more than " + std::to_string(cap) +
            " (use a deeper tree)";
    return HCAPACITY;
  }
  k_sort_segments<<<nleaf, 256, sizeof(int) * (occ > 0 ? occ : 1), st>>>(leaf_start, tmp, h.perm, cap, h.derr); ++h.nlaunch;
  k_gather_points<<<grid, 256, 0, st>>>(soa, h.perm, N, d, soa2); ++h.nlaunch;
  k_check_duplicates<<<nleaf, 128, 0, st>>>(soa2, N, d, leaf_start, h.derr); ++h.nlaunch;
  h.pts = soa2;
  for (int l = 0; l < L; ++l) {
    int nb = 1 << (d * l);
    k_level_starts<<<(nb + 256) / 256, 256, 0, st>>>(leaf_start, d * (L - l), nb, h.start + h.soff[l]); ++h.nlaunch;
  }
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
  int e = check_derr(h);
  if (e == DERR_DUPLICATE) {
    h.err = "duplicate points: the kernel is singular";
    return HINVALID;
  }
  if (e) {
    h.err = "tree build failed (device error " + std::to_string(e) + ")";
    return HCAPACITY;
  }
  double bb[4];
  AIFMM_CUDA_TRY(h, cudaMemcpy(bb, h.bbox, sizeof(bb), cudaMemcpyDeviceToHost));
  if (!(bb[3] > 0.0)) {
    h.err = "degenerate point set (zero extent)";
    return HINVALID;
  }
  return HOK;
}

}  // namespace aifmm
