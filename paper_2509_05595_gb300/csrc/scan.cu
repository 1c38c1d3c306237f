// Deterministic device-wide exclusive prefix sums (reduce / scan-of-sums /
// apply), used for CSR offsets, stream compaction and radix-sort histograms.
#include "common.cuh"

namespace pamo {

namespace {

constexpr int kItems = 8;
constexpr int kTile = kBlock * kItems;  // 2048 items per block

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

template <typename T>
__global__ void k_tile_sums(const T* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t j = base + (int64_t)i * kBlock + threadIdx.x;  // striped: coalesced
    if (j < n) s += (int)in[j];
  }
  s = __reduce_add_sync(0xffffffffu, s);
  __shared__ int ws[kBlock / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kBlock / 32; w++) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// single block: exclusive scan of sums[0..m) in place, total to sums[m]
__global__ void k_scan_sums(int32_t* sums, int64_t m) {
  int carry = 0;
  for (int64_t base = 0; base < m; base += kBlock) {
    int64_t j = base + threadIdx.x;
    int v = j < m ? sums[j] : 0;
    int tot;
    int ex = block_excl_scan(v, tot);
    if (j < m) sums[j] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[m] = carry;
}

template <typename T>
__global__ void k_tile_apply(const T* __restrict__ in, int64_t n, const int32_t* __restrict__ sums,
                             int32_t* __restrict__ out) {
  // blocked arrangement so that each thread owns kItems consecutive items
  __shared__ int32_t tile[kTile];
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
    tile[i * kBlock + threadIdx.x] = j < n ? (int)in[j] : 0;
  }
  __syncthreads();
  int v[kItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    v[i] = tile[threadIdx.x * kItems + i];
    s += v[i];
  }
  int tot;
  int ex = block_excl_scan(s, tot) + sums[blockIdx.x];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    tile[threadIdx.x * kItems + i] = ex;
    ex += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
    if (j < n) out[j] = tile[i * kBlock + threadIdx.x];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    int64_t tiles = gridDim.x;
    out[n] = sums[tiles];
  }
}

template <typename T>
pamo_status scan_impl(const T* in, int32_t* out, int64_t n, Buf& tmp, cudaStream_t st) {
  int64_t tiles = (n + kTile - 1) / kTile;
  if (tiles < 1) tiles = 1;
  PAMO_TRY(buf_reserve(tmp, sizeof(int32_t) * (tiles + 1), st));
  int32_t* sums = (int32_t*)tmp.p;
  k_tile_sums<T><<<(unsigned)tiles, kBlock, 0, st>>>(in, n, sums); note_launch();
  k_scan_sums<<<1, kBlock, 0, st>>>(sums, tiles); note_launch();
  k_tile_apply<T><<<(unsigned)tiles, kBlock, 0, st>>>(in, n, sums, out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace

pamo_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, Buf& tmp,
                               cudaStream_t st) {
  return scan_impl<int32_t>(in, out, n, tmp, st);
}

int64_t scan_sums_count(int64_t n) {
  int64_t tiles = (n + kTile - 1) / kTile;
  return (tiles < 1 ? 1 : tiles) + 1;
}

pamo_status exclusive_scan_i32_into(const int32_t* in, int32_t* out, int64_t n, int32_t* sums,
                                    cudaStream_t st) {
  int64_t tiles = scan_sums_count(n) - 1;
  k_tile_sums<int32_t><<<(unsigned)tiles, kBlock, 0, st>>>(in, n, sums); note_launch();
  k_scan_sums<<<1, kBlock, 0, st>>>(sums, tiles); note_launch();
  k_tile_apply<int32_t><<<(unsigned)tiles, kBlock, 0, st>>>(in, n, sums, out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status exclusive_scan_u8(const uint8_t* in, int32_t* out, int64_t n, Buf& tmp,
                              cudaStream_t st) {
  return scan_impl<uint8_t>(in, out, n, tmp, st);
}

}  // namespace pamo
