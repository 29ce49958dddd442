// validate.cu -- input checks of the CSR contract (Section 3: an undirected weighted graph,
// w_ij = w_ji > 0, stored with both arcs).  Offsets are checked first (the arc checks trust
// them); then targets, weights, the weight total (2m) and symmetry.  Symmetry is tested by a
// signed hash sum: every arc (u -> v, w), u != v, adds +h(min, max, w) if u < v and -h if u > v,
// modulo 2^64, so a symmetric arc multiset sums to zero and any other fails with probability
// 1 - 2^-64.  Results land in ctrl counters; the host turns them into LOUVAIN_ERR_INVALID.
#include "flat.cuh"
#include "internal.cuh"

namespace lv {

__global__ void k_val_offsets(int64_t n, int64_t n_arcs, const int64_t* offs, Ctrl* ctrl) {
  unsigned long long bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (offs[i + 1] < offs[i]) bad++;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (offs[0] != 0 || offs[n] != n_arcs)) bad++;
  if (bad) atomicAdd(&ctrl->cnt[0], bad);
}

void validate_offsets(Ctx& c, int64_t n, int64_t n_arcs, const int64_t* offs, Ctrl* ctrl) {
  k_val_offsets<<<grid_for(n > 0 ? n : 1, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(n, n_arcs, offs, ctrl);
  c.launches++;
}

template <bool FP>
__global__ void __launch_bounds__(kBlock) k_val_arcs(int64_t n, const int64_t* offs, const int32_t* tg, const void* wv,
                                                     Ctrl* ctrl) {
  __shared__ FlatRows fr;
  unsigned long long bad_t = 0, bad_w = 0, sym = 0, isum = 0;
  double fsum = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * kBlock; r0 < n; r0 += (int64_t)gridDim.x * kBlock) {
    const int64_t total = flat_load(fr, r0, n, offs, offs + 1);
    for (int64_t f = threadIdx.x; f < total; f += kBlock) {
      const int row = flat_row(fr, f);
      const int64_t u = r0 + row;
      const int64_t e = fr.beg[row] + (f - fr.excl[row]);
      const int32_t v = tg[e];
      uint32_t wbits;
      if (FP) {
        const float w = reinterpret_cast<const float*>(wv)[e];
        if (!(w > 0.0f) || isinf(w)) bad_w++;
        else fsum += (double)w;
        wbits = __float_as_uint(w);
      } else {
        const int32_t w = reinterpret_cast<const int32_t*>(wv)[e];
        if (w <= 0) bad_w++;
        else isum += (unsigned long long)w;
        wbits = (uint32_t)w;
      }
      if (v < 0 || v >= n) { bad_t++; continue; }
      if (v == u) continue;
      const int64_t lo = u < v ? u : v, hi = u < v ? v : u;
      const uint64_t h = hash3(0x5EEDULL, ((uint64_t)lo << 32) | (uint64_t)hi, wbits);
      sym += u < v ? h : (0ULL - h);
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    bad_t += __shfl_xor_sync(0xffffffffu, bad_t, o);
    bad_w += __shfl_xor_sync(0xffffffffu, bad_w, o);
    sym += __shfl_xor_sync(0xffffffffu, sym, o);
    isum += __shfl_xor_sync(0xffffffffu, isum, o);
    fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad_t) atomicAdd(&ctrl->cnt[1], bad_t);
    if (bad_w) atomicAdd(&ctrl->cnt[2], bad_w);
    if (sym) atomicAdd(&ctrl->cnt[3], sym);
    if (isum) atomicAdd(reinterpret_cast<unsigned long long*>(&ctrl->acc_i[0]), isum);
    if (fsum != 0.0) atomicAdd(&ctrl->acc_f[0], fsum);
  }
}

void validate_arcs(Ctx& c, int64_t n, const int64_t* offs, const int32_t* tg, const void* w, bool fp, Ctrl* ctrl) {
  if (n <= 0) return;
  if (fp) k_val_arcs<true><<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(n, offs, tg, w, ctrl);
  else k_val_arcs<false><<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(n, offs, tg, w, ctrl);
  c.launches++;
}

__global__ void k_val_range(const int32_t* ids, int64_t m, int64_t hi, Ctrl* ctrl) {
  unsigned long long bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (ids[i] < 0 || ids[i] >= hi) bad++;
  if (bad) atomicAdd(&ctrl->cnt[5], bad);
}

void validate_range(Ctx& c, const int32_t* ids, int64_t m, int64_t hi, Ctrl* ctrl) {
  if (m <= 0) return;
  k_val_range<<<grid_for(m, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(ids, m, hi, ctrl);
  c.launches++;
}

__global__ void k_val_reset(Ctrl* c) {
  for (int k = 0; k < 8; k++) c->cnt[k] = 0;
  for (int k = 0; k < 4; k++) { c->acc_i[k] = 0; c->acc_f[k] = 0.0; }
}
void validate_reset(Ctx& c, Ctrl* ctrl) {
  k_val_reset<<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
}

}  // namespace lv
