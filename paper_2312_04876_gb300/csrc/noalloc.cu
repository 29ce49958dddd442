// noalloc.cu -- louvain_exclusive_scan_static: the exclusive scan without any allocation.
//
// Some callers cannot call cudaMalloc: a host application whose memory manager owns all of the
// device memory (a framework's caching allocator, or a fixed HBM budget already handed out), or a
// latency-critical loop that cannot take the implicit device-wide synchronisation of
// cudaMalloc / cudaFree.  For them this entry point runs the same three scan kernels as
// louvain_exclusive_scan, but keeps the scratch (the per-tile sums) in a file-scope __device__
// array instead of a handle's workspace.  Every GPU that loads the library holds that array
// (128 KiB) until the process exits.
#include <mutex>

#include "internal.cuh"

namespace {

// 4096 elements per scan tile (prims.cu); 2^26 elements need 2^14 tile sums (+1 slack).
constexpr int64_t kStaticScanMax = (int64_t)1 << 26;
constexpr int64_t kStaticScanTiles = kStaticScanMax / 4096 + 8;

static __device__ __align__(256) int64_t g_scan_tiles[kStaticScanTiles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t* g_tiles_dev[kMaxDevices] = {};

// Device address of g_scan_tiles on the current device.  In host code the symbol's name is only a
// host-side stand-in, so the address is looked up once per device and cached.
cudaError_t tiles_address(int64_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_tiles_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scan_tiles);
    if (e != cudaSuccess) return e;
    g_tiles_dev[dev] = static_cast<int64_t*>(p);
  }
  *out = g_tiles_dev[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" louvain_status louvain_exclusive_scan_static(const int64_t* d_in, int64_t* d_out, int64_t count,
                                                        void* stream, int64_t* total) {
  if (count < 0 || count > kStaticScanMax || !d_out || (count > 0 && !d_in)) return LOUVAIN_ERR_INVALID;
  int64_t* tiles = nullptr;
  cudaError_t e = tiles_address(&tiles);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LOUVAIN_ERR_CUDA;
  }
  lv::Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  // The tile sums are written in full by the first kernel before the others read them, so
  // nothing left over from an earlier call needs clearing.
  lv::scan_exclusive_i64(c, d_in, d_out, count, tiles);
  if ((e = cudaGetLastError()) != cudaSuccess) return LOUVAIN_ERR_CUDA;
  if (total && (e = cudaMemcpyAsync(total, d_out + count, sizeof(int64_t), cudaMemcpyDeviceToHost, c.s)) != cudaSuccess) {
    cudaGetLastError();
    return LOUVAIN_ERR_CUDA;
  }
  if ((e = cudaStreamSynchronize(c.s)) != cudaSuccess) {
    cudaGetLastError();
    return LOUVAIN_ERR_CUDA;
  }
  return LOUVAIN_OK;
}
