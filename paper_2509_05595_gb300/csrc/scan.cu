// Deterministic device-wide exclusive prefix sums (tile sums / scan of the
// tile sums / apply), used for CSR offsets, stream compaction and radix-sort
// histograms.  The length can come from device memory, so that the scan can
// sit inside a replayed CUDA graph whose sizes change from round to round;
// blocks loop over tiles (grid-stride), so the grid is fixed.  The
// multi-segment form runs up to four independent byte scans (the commit's)
// in one set of three launches over their concatenated tiles.
#include "common.cuh"

namespace pamo {

namespace {

constexpr int kItems = kScanTile / kBlock;
constexpr int kTile = kScanTile;  // 2048 items per tile

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exclusive scan of one value per thread across the block; returns the
// exclusive prefix and the block total
__device__ __forceinline__ int block_excl_scan(int v, int& total) {
  constexpr int NW = kBlock / 32;
  __shared__ int ws[NW + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < NW ? ws[lane] : 0;
    int wi = warp_incl_scan(w);
    if (lane < NW) ws[lane] = wi - w;
    if (lane == NW - 1) ws[NW] = wi;
  }
  __syncthreads();
  int r = ws[wid] + inc - v;
  total = ws[NW];
  __syncthreads();  // ws is reused by the next call
  return r;
}

__device__ __forceinline__ int tiles_of(int n) { return n > 0 ? (n + kTile - 1) / kTile : 1; }

// value of item j: the element itself, or (kNot) 1 for a zero byte
template <typename T, bool kNot>
__device__ __forceinline__ int item(const T* __restrict__ in, int64_t j) {
  return kNot ? (in[j] == 0 ? 1 : 0) : (int)in[j];
}

template <typename T, bool kNot>
__global__ void k_tile_sums(const T* __restrict__ in, const int* n_dev, int n_host,
                            int32_t* __restrict__ sums) {
  const int n = dev_n(n_dev, n_host);
  const int tiles = tiles_of(n);
  __shared__ int ws[kBlock / 32];
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t base = (int64_t)tile * kTile;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t j = base + (int64_t)i * kBlock + threadIdx.x;  // striped: coalesced
      if (j < n) s += item<T, kNot>(in, j);
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < kBlock / 32; w++) t += ws[w];
      sums[tile] = t;
    }
    __syncthreads();
  }
}

// single block: exclusive scan of the tile sums in place, total after them
__global__ void k_scan_sums(int32_t* sums, const int* n_dev, int n_host) {
  const int m = tiles_of(dev_n(n_dev, n_host));
  int carry = 0;
  for (int base = 0; base < m; base += kBlock) {
    const int j = base + threadIdx.x;
    const int v = j < m ? sums[j] : 0;
    int tot;
    const int ex = block_excl_scan(v, tot);
    if (j < m) sums[j] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[m] = carry;
}

template <typename T, bool kNot>
__global__ void k_tile_apply(const T* __restrict__ in, const int* n_dev, int n_host,
                             const int32_t* __restrict__ sums, int32_t* __restrict__ out) {
  // blocked arrangement so that each thread owns kItems consecutive items
  __shared__ int32_t tile_buf[kTile];
  const int n = dev_n(n_dev, n_host);
  const int tiles = tiles_of(n);
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t base = (int64_t)tile * kTile;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
      tile_buf[i * kBlock + threadIdx.x] = j < n ? item<T, kNot>(in, j) : 0;
    }
    __syncthreads();
    int v[kItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      v[i] = tile_buf[threadIdx.x * kItems + i];
      s += v[i];
    }
    int tot;
    int ex = block_excl_scan(s, tot) + sums[tile];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      tile_buf[threadIdx.x * kItems + i] = ex;
      ex += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
      if (j < n) out[j] = tile_buf[i * kBlock + threadIdx.x];
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[tiles];
}

template <typename T, bool kNot = false>
pamo_status scan_launch(const T* in, const int* n_dev, int n_host, int32_t* out, int32_t* sums,
                        int grid, cudaStream_t st) {
  k_tile_sums<T, kNot><<<grid, kBlock, 0, st>>>(in, n_dev, n_host, sums); note_launch();
  k_scan_sums<<<1, kBlock, 0, st>>>(sums, n_dev, n_host); note_launch();
  k_tile_apply<T, kNot><<<grid, kBlock, 0, st>>>(in, n_dev, n_host, sums, out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

struct ScanSegs {
  ScanSeg s[kMaxScanSegs];
  int count;
};

__device__ __forceinline__ int seg_item(const ScanSeg& g, int64_t j) {
  const int v = g.in[g.gather ? (int64_t)g.gather[j] : j];
  return g.invert ? (v == 0 ? 1 : 0) : v;
}

// tile t of the concatenated tile index space -> (segment, local tile)
__device__ __forceinline__ int seg_of(const ScanSegs& g, int t, int& local, int& total) {
  int k = -1;
  total = 0;
  for (int q = 0; q < g.count; q++) {
    const int m = tiles_of(*g.s[q].n);
    if (k < 0 && t < total + m) {
      k = q;
      local = t - total;
    }
    total += m;
  }
  return k;
}

__global__ void k_multi_tile_sums(ScanSegs g) {
  __shared__ int ws[kBlock / 32];
  int local = 0, total = 0;
  seg_of(g, 0, local, total);
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int lt = 0, tt = 0;
    const ScanSeg& sg = g.s[seg_of(g, tile, lt, tt)];
    const int n = *sg.n;
    const int64_t base = (int64_t)lt * kTile;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
      if (j < n) s += seg_item(sg, j);
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < kBlock / 32; w++) t += ws[w];
      sg.sums[lt] = t;
    }
    __syncthreads();
  }
}

// single block: each segment's tile sums scanned in place, its total after them
__global__ void k_multi_scan_sums(ScanSegs g) {
  for (int q = 0; q < g.count; q++) {
    int32_t* sums = g.s[q].sums;
    const int m = tiles_of(*g.s[q].n);
    int carry = 0;
    for (int base = 0; base < m; base += kBlock) {
      const int j = base + threadIdx.x;
      const int v = j < m ? sums[j] : 0;
      int tot;
      const int ex = block_excl_scan(v, tot);
      if (j < m) sums[j] = carry + ex;
      carry += tot;
    }
    if (threadIdx.x == 0) sums[m] = carry;
  }
}

__global__ void k_multi_tile_apply(ScanSegs g) {
  __shared__ int32_t tile_buf[kTile];
  int local = 0, total = 0;
  seg_of(g, 0, local, total);
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int lt = 0, tt = 0;
    const ScanSeg& sg = g.s[seg_of(g, tile, lt, tt)];
    const int n = *sg.n;
    const int64_t base = (int64_t)lt * kTile;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
      tile_buf[i * kBlock + threadIdx.x] = j < n ? seg_item(sg, j) : 0;
    }
    __syncthreads();
    int v[kItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      v[i] = tile_buf[threadIdx.x * kItems + i];
      s += v[i];
    }
    int tot;
    int ex = block_excl_scan(s, tot) + sg.sums[lt];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      tile_buf[threadIdx.x * kItems + i] = ex;
      ex += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
      if (j < n) sg.out[j] = tile_buf[i * kBlock + threadIdx.x];
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x < g.count) {
    const ScanSeg& sg = g.s[threadIdx.x];
    const int n = *sg.n;
    sg.out[n] = sg.sums[tiles_of(n)];
  }
}

}  // namespace

int64_t scan_sums_count(int64_t n) {
  int64_t tiles = (n + kTile - 1) / kTile;
  return (tiles < 1 ? 1 : tiles) + 1;
}

pamo_status scan_dev_i32(const int32_t* in, const int* n_dev, int32_t* out, int32_t* sums, int grid,
                         cudaStream_t st) {
  return scan_launch<int32_t>(in, n_dev, 0, out, sums, grid, st);
}

pamo_status scan_dev_u8(const uint8_t* in, const int* n_dev, int32_t* out, int32_t* sums, int grid,
                        cudaStream_t st) {
  return scan_launch<uint8_t>(in, n_dev, 0, out, sums, grid, st);
}

pamo_status scan_dev_u8_multi(const ScanSeg* segs, int count, int grid, cudaStream_t st) {
  if (count < 1 || count > kMaxScanSegs) {
    set_error("scan_dev_u8_multi: 1 to 4 segments");
    return PAMO_EINTERNAL;
  }
  ScanSegs g;
  for (int q = 0; q < count; q++) g.s[q] = segs[q];
  g.count = count;
  k_multi_tile_sums<<<grid, kBlock, 0, st>>>(g); note_launch();
  k_multi_scan_sums<<<1, kBlock, 0, st>>>(g); note_launch();
  k_multi_tile_apply<<<grid, kBlock, 0, st>>>(g); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
