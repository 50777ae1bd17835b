// Kernels of the learned warm-start network (a small 3-D U-Net on one coarse
// multigrid level).  Activations are channels-last BF16 ([voxel][channel]);
// convolutions are implicit GEMMs on the BF16 tensor cores with FP32
// accumulation (mma.sync m16n8k16): M = voxels (16 per warp), N = output
// channels, K = 27 taps x input channels, split over three warps per voxel tile.  3x3x3 stencils are periodic in x
// and y and zero-padded in z, like the device.  Gradients with respect to the
// input use the same kernel with the taps flipped and the channel matrices
// transposed (the adjoint convolution); gradients with respect to the weights
// contract over voxels (M = input channels, N = output channels, K = voxels)
// and are summed into FP32 with atomics.  Master weights, Adam moments and
// gradients are FP32; the kernels read BF16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ferrox_internal.cuh"

namespace fx {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// voxel index of the neighbour at tap (dz, dy, dx) = (tap/9, tap/3%3, tap%3) - 1,
// or -1 outside the z range
__device__ __forceinline__ int nb_index(int z, int y, int x, int tap, const NNGrid& g) {
  const int zz = z + tap / 9 - 1;
  if (zz < 0 || zz >= g.D) return -1;
  int yy = y + (tap / 3) % 3 - 1;
  yy = yy < 0 ? yy + g.H : (yy >= g.H ? yy - g.H : yy);
  int xx = x + tap % 3 - 1;
  xx = xx < 0 ? xx + g.W : (xx >= g.W ? xx - g.W : xx);
  return (zz * g.H + yy) * g.W + xx;
}

__device__ __forceinline__ void voxel_zyx(int m, const NNGrid& g, int& z, int& y, int& x) {
  const int hw = g.H * g.W;
  z = m / hw;
  const int r = m - z * hw;
  y = r / g.W;
  x = r - y * g.W;
}

// out[m][co] = act(bias[co] + sum_tap sum_ci in[nb(m, tap)][ci] w[tap][ci][co]),
// weights in the kernel layout wk[tap][co][ci] (BF16).  A block holds kConvTiles
// tiles of 16 voxels; the three warps of a tile (threadIdx.z) split the 27 taps
// by z offset (9 each), so every warp's chain of dependent gathers is one slab,
// and the partial sums meet in shared memory in a fixed order (slab 0 + slab 1
// + slab 2).
constexpr int kConvTiles = 4;

template <int COUT>
__global__ void __launch_bounds__(32 * kConvTiles * 3) conv_fwd_kernel(
    const bf16* __restrict__ in, int cin, const bf16* __restrict__ wk,
    const float* __restrict__ bias, NNGrid g, int relu, bf16* __restrict__ out_bf,
    float* __restrict__ out_f, int f_ch0) {
  __shared__ float part[2][kConvTiles][COUT / 8][4][32];
  const int lane = threadIdx.x, tile = threadIdx.y, slab = threadIdx.z;
  const int M = g.D * g.H * g.W;
  const int m0 = (blockIdx.x * kConvTiles + tile) * 16;
  const bool active = m0 < M;
  const int gq = lane >> 2, tq = lane & 3;
  int zr[2], yr[2], xr[2];
  bool val[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int m = m0 + gq + 8 * r;
    val[r] = m < M;
    voxel_zyx(val[r] ? m : 0, g, zr[r], yr[r], xr[r]);
  }
  float acc[COUT / 8][4];
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  const unsigned* inw = reinterpret_cast<const unsigned*>(in);
  const unsigned* ww = reinterpret_cast<const unsigned*>(wk);
  const int cin2 = cin >> 1;
  if (active) {
    // the slab's nine taps unrolled: their gathers are all in flight before the
    // MMAs that consume them (the layer is latency-bound at these sizes)
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int tap = slab * 9 + t;
      const int n0 = val[0] ? nb_index(zr[0], yr[0], xr[0], tap, g) : -1;
      const int n1 = val[1] ? nb_index(zr[1], yr[1], xr[1], tap, g) : -1;
      for (int c0 = 0; c0 < cin; c0 += 16) {
        const int off = (c0 >> 1) + tq;
        unsigned a[4];
        a[0] = n0 >= 0 ? __ldg(inw + (size_t)n0 * cin2 + off) : 0u;
        a[1] = n1 >= 0 ? __ldg(inw + (size_t)n1 * cin2 + off) : 0u;
        a[2] = n0 >= 0 ? __ldg(inw + (size_t)n0 * cin2 + off + 4) : 0u;
        a[3] = n1 >= 0 ? __ldg(inw + (size_t)n1 * cin2 + off + 4) : 0u;
#pragma unroll
        for (int j = 0; j < COUT / 8; ++j) {
          const unsigned* wp = ww + (size_t)(tap * COUT + j * 8 + gq) * cin2 + off;
          const unsigned b[2] = {__ldg(wp), __ldg(wp + 4)};
          mma_bf16(acc[j], a, b);
        }
      }
    }
  }
  if (slab > 0) {
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) part[slab - 1][tile][j][q][lane] = acc[j][q];
  }
  __syncthreads();
  if (slab > 0 || !active) return;
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = (acc[j][q] + part[0][tile][j][q][lane]) + part[1][tile][j][q][lane];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (!val[r]) continue;
    const int m = m0 + gq + 8 * r;
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j) {
      const int co = j * 8 + 2 * tq;
      float v0 = acc[j][2 * r], v1 = acc[j][2 * r + 1];
      if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
      if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
      if (out_bf)
        *reinterpret_cast<__nv_bfloat162*>(out_bf + (size_t)m * COUT + co) = __floats2bfloat162_rn(v0, v1);
      if (out_f && f_ch0) {
        if (co == 0) out_f[m] = v0;
      } else if (out_f) {
        out_f[(size_t)m * COUT + co] = v0;
        out_f[(size_t)m * COUT + co + 1] = v1;
      }
    }
  }
}

// ---- 3x3x3 convolution on the fifth-generation tensor cores (tcgen05, TMEM) ----------
//
// A tile is 8 (x) x 16 (y) x zt (z) voxels.  Its input with a one-voxel halo
// (10 x 18 x (zt + 2) voxels, periodic in x and y, zero outside z) is staged in
// shared memory in the no-swizzle K-major layout of the tensor core's operands:
// for each 8-channel chunk a plane of 16-byte entries [z][y][x].  Eight
// consecutive x voxels are then one 8 x 16 B core matrix and the 16 y rows of a
// tile are core matrices 160 B apart, so the A operand of every tap is the same
// staged tile seen through a shifted descriptor: the 27 taps need no further
// data movement.  The weights of all taps sit beside it as [tap][ci/8][co][ci%8].
// One thread issues the 128 x COUT x 16 MMAs (27 taps x CIN/16 K-steps per
// z-plane) into FP32 accumulators in tensor memory; the four warps read their
// 32 rows back with tcgen05.ld for the bias, ReLU and BF16/FP32 store.
//
// CTAs are persistent: the weights are loaded once, and the halo buffers and
// accumulators are double-buffered, so the loads of tile i + 1 and the epilogue
// of tile i - 1 run while the tensor core works on tile i.
constexpr int kTcX = 8, kTcY = 16, kTcHX = kTcX + 2, kTcHY = kTcY + 2;
constexpr int kTcPlane = kTcHX * kTcHY;             // halo entries per z-plane
constexpr int kTcThreads = 128;
constexpr long long kTcWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tc_cp16(unsigned dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (8-row group) byte offsets, descriptor version 1, no swizzle.  The start
// address is the low field (bits 0-13, in 16-byte units), so a descriptor of an
// address 16 k bytes further is this one plus k.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n
__host__ __device__ constexpr unsigned tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned mbar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait on an mbarrier phase; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try(mbar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// 16 consecutive FP32 accumulator columns of this warp's 32 rows
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__host__ __device__ constexpr int tc_cols(int n) {
  return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512;
}

struct TcTile {
  int x0, y0, z0;
};

__device__ __forceinline__ TcTile tc_tile(int t, const NNGrid& g, int zt) {
  const int nbx = g.W / kTcX, nby = g.H / kTcY;
  return TcTile{(t % nbx) * kTcX, ((t / nbx) % nby) * kTcY, (t / (nbx * nby)) * zt};
}

// Stage the halo of one tile: warp w takes halo rows (z, y) w, w + 4, ...; lane j
// takes entries j and j + 32 of a row, entry q = x * NCH + chunk, so a warp reads
// consecutive 16-byte chunks of consecutive voxels.  With UP the 48 input
// channels are the concatenation [up(a4) (32), s1 (16)] read in place: chunks
// 0-3 from the coarse field a4 (= in) at the parent voxel, chunks 4-5 from s1.
template <int CIN, bool UP>
__device__ __forceinline__ void tc_load_halo(const bf16* __restrict__ in, const bf16* __restrict__ s1,
                                             const NNGrid& g, TcTile t, int zt, unsigned buf, int chunk_entries) {
  constexpr int NCH = CIN / 8, PER_ROW = kTcHX * NCH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Hc = g.H / 2, Wc = g.W / 2;
  int goff[2], soff[2];
  bool have[2], fine[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = lane + 32 * h;
    have[h] = q < PER_ROW;
    const int xx = have[h] ? q / NCH : 0, k = q % NCH;
    int gx = t.x0 + xx - 1;
    gx = gx < 0 ? gx + g.W : (gx >= g.W ? gx - g.W : gx);
    fine[h] = !UP || k >= 4;
    goff[h] = UP ? (k < 4 ? (gx >> 1) * 32 + 8 * k : gx * 16 + 8 * (k - 4)) : gx * CIN + 8 * k;
    soff[h] = 16 * (k * chunk_entries + xx);
  }
  const int rows = kTcHY * (zt + 2);
  for (int r = warp; r < rows; r += kTcThreads / 32) {
    const int zz = r / kTcHY, yy = r - zz * kTcHY;
    int gy = t.y0 + yy - 1;
    gy = gy < 0 ? gy + g.H : (gy >= g.H ? gy - g.H : gy);
    int gz = t.z0 + zz - 1;
    const bool okz = gz >= 0 && gz < g.D;
    gz = okz ? gz : 0;
    const bf16* row = UP ? s1 + (size_t)(gz * g.H + gy) * g.W * 16 : in + (size_t)(gz * g.H + gy) * g.W * CIN;
    const bf16* crow = UP ? in + (size_t)((gz >> 1) * Hc + (gy >> 1)) * Wc * 32 : row;
    const unsigned srow = buf + 16u * (unsigned)(r * kTcHX);
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (have[h]) tc_cp16(srow + soff[h], (fine[h] ? row : crow) + goff[h], okz);
  }
}

template <int CIN, int COUT>
__device__ __forceinline__ void tc_epilogue(unsigned tmem_acc, const NNGrid& g, TcTile t, int zt,
                                            const float* __restrict__ bias, int relu, bf16* __restrict__ out_bf,
                                            float* __restrict__ out_f, int f_ch0) {
  const int tid = threadIdx.x, warp = tid >> 5;
  // thread tid holds accumulator row tid = voxel (y0 + tid / 8, x0 + tid % 8)
  const int x = t.x0 + (tid & 7), y = t.y0 + (tid >> 3);
  for (int p = 0; p < zt; ++p) {
    const size_t m = ((size_t)(t.z0 + p) * g.H + y) * g.W + x;
#pragma unroll
    for (int j = 0; j < COUT / 16; ++j) {
      float v[16];
      tc_ld16(tmem_acc + ((unsigned)(32 * warp) << 16) + (unsigned)(p * COUT + 16 * j), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (bias) v[i] += __ldg(bias + 16 * j + i);
        if (relu) v[i] = fmaxf(v[i], 0.f);
      }
      if (out_bf) {
        uint4 q[2];
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(q);
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        uint4* o = reinterpret_cast<uint4*>(out_bf + m * COUT + 16 * j);
        o[0] = q[0];
        o[1] = q[1];
      }
      if (out_f && f_ch0) {
        if (j == 0) out_f[m] = v[0];
      } else if (out_f) {
        float4* o = reinterpret_cast<float4*>(out_f + m * COUT + 16 * j);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    }
  }
}

template <int CIN, int COUT, bool UP>
__global__ void __launch_bounds__(kTcThreads) conv_tc_kernel(
    const bf16* __restrict__ in, const bf16* __restrict__ s1, const bf16* __restrict__ wt,
    const float* __restrict__ bias, NNGrid g, int zt, int relu, bf16* __restrict__ out_bf,
    float* __restrict__ out_f, int f_ch0, int* __restrict__ fault) {
  constexpr int NCH = CIN / 8;
  constexpr int WBYTES = 27 * CIN * COUT * 2;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem);   // two barriers
  unsigned* tslot = reinterpret_cast<unsigned*>(smem + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ncols = tc_cols(2 * zt * COUT);
  const int chunk_entries = kTcPlane * (zt + 2);
  const unsigned hbytes = 16u * NCH * chunk_entries;
  const unsigned sw = smem_u32(smem + 128);
  const unsigned hb0 = sw + WBYTES, mb0 = smem_u32(mbar);   // buffer / barrier b at + b hbytes / + 8 b
  const int ntiles = (g.W / kTcX) * (g.H / kTcY) * (g.D / zt);
  const int nmine = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // weights (a straight copy of the packed array) and the first tile, one group
  for (int i = tid; i < WBYTES / 16; i += kTcThreads) tc_cp16(sw + 16u * i, wt + 8 * i, true);
  if (nmine > 0) tc_load_halo<CIN, UP>(in, s1, g, tc_tile(blockIdx.x, g, zt), zt, hb0, chunk_entries);
  asm volatile("cp.async.commit_group;\n" ::: "memory");

  constexpr unsigned idesc = tc_idesc(COUT);
  const unsigned a_lbo = 16u * chunk_entries, b_lbo = 16u * COUT;
  const unsigned long long bdesc0 = tc_desc(sw, b_lbo, 128u);
  unsigned tmem = 0;
  bool ok = true;
  int issued = 0;   // tiles whose MMAs were committed
  for (int i = 0; i < nmine; ++i) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    ok = !__syncthreads_or(!ok);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) break;
    tmem = *tslot;
    const int cur = i & 1;
    if (tid == 0) {
      const unsigned d0 = tmem + (unsigned)(cur * zt * COUT);
      const unsigned long long adesc0 = tc_desc(hb0 + cur * hbytes, a_lbo, 16u * kTcHX);
      const unsigned long long kstep = 2ull * (unsigned long long)chunk_entries;   // 16-byte units
      for (int p = 0; p < zt; ++p) {
        const unsigned long long ap = adesc0 + (unsigned long long)(p * kTcPlane);
#pragma unroll 3
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          const unsigned long long at = ap + (unsigned long long)((dz * kTcHY + dy) * kTcHX + dx);
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ++ks)
            tc_mma(d0 + (unsigned)(p * COUT), at + ks * kstep,
                   bdesc0 + (unsigned long long)((tap * NCH + 2 * ks) * COUT), idesc, (tap | ks) != 0);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb0 + 8 * cur)
                   : "memory");
    }
    issued = i + 1;
    __syncwarp();
    if (i > 0) {   // tile i - 1: its MMAs done frees its halo buffer and accumulator
      ok = __all_sync(0xffffffffu, mbar_wait(mb0 + 8 * (cur ^ 1), ((i - 1) >> 1) & 1, kTcWaitCycles));
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (ok && i + 1 < nmine)
      tc_load_halo<CIN, UP>(in, s1, g, tc_tile(blockIdx.x + (i + 1) * gridDim.x, g, zt), zt,
                            hb0 + (cur ^ 1) * hbytes, chunk_entries);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (ok && i > 0)
      tc_epilogue<CIN, COUT>(tmem + (unsigned)((cur ^ 1) * zt * COUT), g, tc_tile(blockIdx.x + (i - 1) * gridDim.x, g, zt),
                             zt, bias, relu, out_bf, out_f, f_ch0);
  }
  if (ok && nmine > 0) {
    const int l = nmine - 1;
    ok = __all_sync(0xffffffffu, mbar_wait(mb0 + 8 * (l & 1), (l >> 1) & 1, kTcWaitCycles));
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok)
      tc_epilogue<CIN, COUT>(tmem + (unsigned)((l & 1) * zt * COUT), g, tc_tile(blockIdx.x + l * gridDim.x, g, zt), zt,
                             bias, relu, out_bf, out_f, f_ch0);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (!ok && tid == 0) {
    atomicExch(fault, 1);
    // let the last committed MMAs drain before the columns are freed
    if (issued > 0) mbar_wait(mb0 + 8 * ((issued - 1) & 1), ((issued - 1) >> 1) & 1, kTcWaitCycles);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned base = *tslot;
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(ncols) : "memory");
  }
}

// gw[tap][ci][co] += sum_m in[nb(m, tap)][ci] dout[m][co] over this warp's voxel chunk
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) conv_wgrad_kernel(const bf16* __restrict__ in,
                                                         const bf16* __restrict__ dout, NNGrid g,
                                                         int chunk, float* __restrict__ gw) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int M = g.D * g.H * g.W;
  const int nparts = (M + chunk - 1) / chunk;
  if (warp >= 27 * nparts) return;
  const int tap = warp % 27, part = warp / 27;
  const int mb = part * chunk, me = min(M, mb + chunk);
  const int gq = lane >> 2, tq = lane & 3;
  float acc[CIN / 16][COUT / 8][4];
#pragma unroll
  for (int c = 0; c < CIN / 16; ++c)
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j) acc[c][j][0] = acc[c][j][1] = acc[c][j][2] = acc[c][j][3] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int m0 = mb; m0 < me; m0 += 16) {
    // the four voxels of this thread's K slots: 2tq, 2tq+1, 2tq+8, 2tq+9
    int nbv[4];
    bool okv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + 2 * tq + (q & 1) + 8 * (q >> 1);
      okv[q] = m < me;
      int z, y, x;
      voxel_zyx(okv[q] ? m : 0, g, z, y, x);
      nbv[q] = okv[q] ? nb_index(z, y, x, tap, g) : -1;
    }
    unsigned bfr[COUT / 8][2];
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j) {
      const int co = j * 8 + gq;
      bf16 d[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + 2 * tq + (q & 1) + 8 * (q >> 1);
        d[q] = okv[q] ? dout[(size_t)m * COUT + co] : zero;
      }
      bfr[j][0] = pack2(d[0], d[1]);
      bfr[j][1] = pack2(d[2], d[3]);
    }
#pragma unroll
    for (int c = 0; c < CIN / 16; ++c) {
      bf16 lo[4], hi[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        lo[q] = nbv[q] >= 0 ? in[(size_t)nbv[q] * CIN + c * 16 + gq] : zero;
        hi[q] = nbv[q] >= 0 ? in[(size_t)nbv[q] * CIN + c * 16 + gq + 8] : zero;
      }
      const unsigned a[4] = {pack2(lo[0], lo[1]), pack2(hi[0], hi[1]), pack2(lo[2], lo[3]),
                             pack2(hi[2], hi[3])};
#pragma unroll
      for (int j = 0; j < COUT / 8; ++j) mma_bf16(acc[c][j], a, bfr[j]);
    }
  }
#pragma unroll
  for (int c = 0; c < CIN / 16; ++c)
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j) {
      float* base = gw + (size_t)tap * CIN * COUT;
      const int co = j * 8 + 2 * tq;
      atomicAdd(base + (c * 16 + gq) * COUT + co, acc[c][j][0]);
      atomicAdd(base + (c * 16 + gq) * COUT + co + 1, acc[c][j][1]);
      atomicAdd(base + (c * 16 + gq + 8) * COUT + co, acc[c][j][2]);
      atomicAdd(base + (c * 16 + gq + 8) * COUT + co + 1, acc[c][j][3]);
    }
}

__global__ void bias_grad_kernel(const bf16* __restrict__ dout, int M, int C, int chunk, float* gb) {
  const int c = threadIdx.x % C;
  const int part = blockIdx.x * (blockDim.x / C) + threadIdx.x / C;
  if (threadIdx.x >= (blockDim.x / C) * C) return;
  float s = 0.f;
  for (int m = part * chunk; m < min(M, (part + 1) * chunk); ++m) s += __bfloat162float(dout[(size_t)m * C + c]);
  atomicAdd(gb + c, s);
}

// 2x2x2 mean of a fine channels-last field: one thread per coarse voxel and
// 8-channel chunk (16 bytes)
__global__ void pool2_kernel(const bf16* __restrict__ in, NNGrid f, int C, bf16* __restrict__ out) {
  const int Dc = f.D / 2, Hc = f.H / 2, Wc = f.W / 2, nch = C / 8;
  const long long n = (long long)Dc * Hc * Wc * nch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % nch);
    const long long v = t / nch;
    const int X = (int)(v % Wc), Y = (int)((v / Wc) % Hc), Z = (int)(v / ((long long)Wc * Hc));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < 8; ++q) {
      const int z = 2 * Z + (q >> 2), y = 2 * Y + ((q >> 1) & 1), x = 2 * X + (q & 1);
      const uint4 u = *reinterpret_cast<const uint4*>(in + ((size_t)(z * f.H + y) * f.W + x) * C + 8 * k);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 p = __bfloat1622float2(h[i]);
        s[2 * i] += p.x;
        s[2 * i + 1] += p.y;
      }
    }
    uint4 o;
    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int i = 0; i < 4; ++i) oh[i] = __floats2bfloat162_rn(0.125f * s[2 * i], 0.125f * s[2 * i + 1]);
    *reinterpret_cast<uint4*>(out + (size_t)v * C + 8 * k) = o;
  }
}

// cat[v] = [a4(parent of v) (32 channels), s1(v) (16 channels)]: one thread per
// voxel and 8-channel chunk (16 bytes)
__global__ void upcat_kernel(const bf16* __restrict__ a4, const bf16* __restrict__ s1, NNGrid f,
                             bf16* __restrict__ cat) {
  const long long n = (long long)f.D * f.H * f.W * 6;
  const int Hc = f.H / 2, Wc = f.W / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % 6);
    const long long v = t / 6;
    const int x = (int)(v % f.W), y = (int)((v / f.W) % f.H), z = (int)(v / ((long long)f.W * f.H));
    const uint4 u = k < 4 ? *reinterpret_cast<const uint4*>(a4 + ((size_t)((z / 2) * Hc + y / 2) * Wc + x / 2) * 32 + 8 * k)
                          : *reinterpret_cast<const uint4*>(s1 + (size_t)v * 16 + 8 * (k - 4));
    *reinterpret_cast<uint4*>(cat + (size_t)v * 48 + 8 * k) = u;
  }
}

// out = bf16(d * (act > 0))   (ReLU backward; act is the post-activation)
__global__ void mask_kernel(const float* __restrict__ d, const bf16* __restrict__ act, long long n,
                            bf16* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = __float2bfloat16(__bfloat162float(act[t]) > 0.f ? d[t] : 0.f);
}

// da4m[V][c] = bf16(sum over the 8 children of dcat[child][c] (c < 32), masked by a4 > 0)
__global__ void up_grad_kernel(const float* __restrict__ dcat, const bf16* __restrict__ a4, NNGrid f,
                               bf16* __restrict__ out) {
  const int Dc = f.D / 2, Hc = f.H / 2, Wc = f.W / 2;
  const long long n = (long long)Dc * Hc * Wc * 32;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % 32);
    const long long v = t / 32;
    const int X = (int)(v % Wc), Y = (int)((v / Wc) % Hc), Z = (int)(v / ((long long)Wc * Hc));
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int z = 2 * Z + (q >> 2), y = 2 * Y + ((q >> 1) & 1), x = 2 * X + (q & 1);
      s += dcat[((size_t)(z * f.H + y) * f.W + x) * 48 + c];
    }
    out[t] = __float2bfloat16(__bfloat162float(a4[t]) > 0.f ? s : 0.f);
  }
}

// ds1m[v][c] = bf16((dcat[v][32 + c] + dp[parent(v)][c] / 8) masked by s1 > 0)
__global__ void skip_grad_kernel(const float* __restrict__ dcat, const float* __restrict__ dp,
                                 const bf16* __restrict__ s1, NNGrid f, bf16* __restrict__ out) {
  const long long n = (long long)f.D * f.H * f.W * 16;
  const int Hc = f.H / 2, Wc = f.W / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % 16);
    const long long v = t / 16;
    const int x = (int)(v % f.W), y = (int)((v / f.W) % f.H), z = (int)(v / ((long long)f.W * f.H));
    const float g = dcat[(size_t)v * 48 + 32 + c] +
                    0.125f * dp[((size_t)((z / 2) * Hc + y / 2) * Wc + x / 2) * 16 + c];
    out[t] = __float2bfloat16(__bfloat162float(s1[t]) > 0.f ? g : 0.f);
  }
}

// loss += sum (y0 - t)^2 / M; dy[m][0] = 2 (y0 - t) / M, other channels 0
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ tgt, int M,
                           bf16* __restrict__ dy, float* __restrict__ loss) {
  float s = 0.f;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    const float d = y[m] - tgt[m];
    s += d * d;
    dy[(size_t)m * 16] = __float2bfloat16(2.f * d / M);
    for (int c = 1; c < 16; ++c) dy[(size_t)m * 16 + c] = __float2bfloat16(0.f);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / M);
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float c1,
                            float c2, float eps) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const float gr = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gr;
    const float vt = b2 * v[t] + (1.f - b2) * gr * gr;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    g[t] = 0.f;
  }
}

// kernel layouts from the FP32 master [tap][ci][co]: forward wk[tap][co][ci];
// adjoint wb[tap][ci][co] = w[26 - tap][ci][co] read as a conv with Cin' = co, Cout' = ci;
// the same two in the tensor-memory kernel's operand layout [tap][cin/8][cout][cin%8]:
// wkt for the forward, wbt (Cin' = co, Cout' = ci) for the adjoint
__global__ void pack_kernel(const float* __restrict__ w, int cin, int cout, bf16* __restrict__ wk,
                            bf16* __restrict__ wb, bf16* __restrict__ wkt, bf16* __restrict__ wbt) {
  const int n = 27 * cin * cout;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int co = t % cout, ci = (t / cout) % cin, tap = t / (cin * cout);
    const bf16 val = __float2bfloat16(w[t]);
    wk[((size_t)tap * cout + co) * cin + ci] = val;
    wb[((size_t)(26 - tap) * cin + ci) * cout + co] = val;
    wkt[(((size_t)tap * (cin / 8) + ci / 8) * cout + co) * 8 + ci % 8] = val;
    wbt[(((size_t)(26 - tap) * (cout / 8) + co / 8) * cin + ci) * 8 + co % 8] = val;
  }
}

int grid1(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 8) b = 152LL * 8;
  return (int)(b < 1 ? 1 : b);
}

// dynamic shared memory of a tensor-memory CTA (barriers, weights, two halo
// buffers), padded so that the CTAs that fit on one SM never ask for more than
// its 512 tensor-memory columns together
size_t tc_smem(int cin, int cout, int zt) {
  const size_t b = 128 + (size_t)27 * cin * cout * 2 + 2 * (size_t)(cin / 8) * kTcPlane * (zt + 2) * 16;
  const int per_sm = 512 / tc_cols(2 * zt * cout);
  const size_t floor_b = 233472 / (per_sm + 1) - 1024 + 16;
  return std::max(b, floor_b);
}

int tc_tiles(NNGrid g, int zt) { return (g.W / kTcX) * (g.H / kTcY) * (g.D / zt); }

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n < 1) n = 1;
  }
  return n;
}

// z-planes per tile: the most of {4, 2} that divides D, fits the shared memory
// and still gives every SM a tile, else 1
int tc_zt(int cin, int cout, NNGrid g) {
  for (int zt : {4, 2})
    if (g.D % zt == 0 && tc_smem(cin, cout, zt) <= 232448 && tc_tiles(g, zt) >= sm_count()) return zt;
  return 1;
}

template <int CIN, int COUT, bool UP = false>
void launch_conv_tc(const bf16* in, const bf16* s1, const bf16* wt, const float* bias, NNGrid g, int relu,
                    bf16* out_bf, float* out_f, int f_ch0, int* fault, cudaStream_t s) {
  const int zt = tc_zt(CIN, COUT, g);
  const size_t smem = tc_smem(CIN, COUT, zt);
  const int per_sm = std::max(1, std::min(16, (int)(233472 / (smem + 1024))));
  const int blocks = std::min(tc_tiles(g, zt), sm_count() * per_sm);
  conv_tc_kernel<CIN, COUT, UP><<<blocks, kTcThreads, smem, s>>>(in, s1, wt, bias, g, zt, relu, out_bf, out_f,
                                                                    f_ch0, fault);
}

}  // namespace

// Shared-memory limits of the tensor-memory kernels, set once per process when
// a network is created, so that no launch (possibly inside a stream capture)
// has to configure its function first.
cudaError_t nn_tc_setup() {
  static cudaError_t done = [] {
    const int lim = 232448;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
      const cudaError_t r = cudaFuncSetAttribute(f, a, lim);
      if (e == cudaSuccess) e = r;
    };
    set((const void*)conv_tc_kernel<16, 16, false>);
    set((const void*)conv_tc_kernel<16, 32, false>);
    set((const void*)conv_tc_kernel<16, 48, false>);
    set((const void*)conv_tc_kernel<32, 16, false>);
    set((const void*)conv_tc_kernel<32, 32, false>);
    set((const void*)conv_tc_kernel<48, 16, false>);
    set((const void*)conv_tc_kernel<48, 16, true>);
    return e;
  }();
  return done;
}

// The tensor-memory kernel takes grids whose x extent is a multiple of 8 and y
// extent a multiple of 16; other grids use the mma.sync kernel.
bool nn_conv_uses_tc(int cin, int cout, NNGrid g) {
  if (g.W % kTcX || g.H % kTcY || g.D < 1) return false;
  return (cin == 16 && (cout == 16 || cout == 32 || cout == 48)) || (cin == 32 && (cout == 16 || cout == 32)) ||
         (cin == 48 && cout == 16);
}

bool nn_conv_fwd(const bf16* in, int cin, const bf16* wk, const bf16* wt, const float* bias, int cout,
                 NNGrid g, int relu, bf16* out_bf, float* out_f, int f_ch0, int* fault, cudaStream_t s) {
  if (wt && fault && nn_conv_uses_tc(cin, cout, g)) {
    auto go = [&](auto launch) { launch(in, nullptr, wt, bias, g, relu, out_bf, out_f, f_ch0, fault, s); };
    if (cin == 16 && cout == 16) go(launch_conv_tc<16, 16>);
    else if (cin == 16 && cout == 32) go(launch_conv_tc<16, 32>);
    else if (cin == 16 && cout == 48) go(launch_conv_tc<16, 48>);
    else if (cin == 32 && cout == 16) go(launch_conv_tc<32, 16>);
    else if (cin == 32 && cout == 32) go(launch_conv_tc<32, 32>);
    else go(launch_conv_tc<48, 16>);
    return true;
  }
  const int M = g.D * g.H * g.W;
  const int tiles = (M + 15) / 16;
  const int blocks = (tiles + kConvTiles - 1) / kConvTiles;
  const dim3 block(32, kConvTiles, 3);
  if (cout == 16) conv_fwd_kernel<16><<<blocks, block, 0, s>>>(in, cin, wk, bias, g, relu, out_bf, out_f, f_ch0);
  else if (cout == 32) conv_fwd_kernel<32><<<blocks, block, 0, s>>>(in, cin, wk, bias, g, relu, out_bf, out_f, f_ch0);
  else if (cout == 48) conv_fwd_kernel<48><<<blocks, block, 0, s>>>(in, cin, wk, bias, g, relu, out_bf, out_f, f_ch0);
  return false;
}

// conv(48 -> 16) of [up(a4), s1] on the tensor-memory kernel without forming the
// concatenation; false (nothing launched) where the grid does not allow it
bool nn_conv_upcat_tc(const bf16* a4, const bf16* s1, const bf16* wt, const float* bias, NNGrid g, int relu,
                      bf16* out_bf, int* fault, cudaStream_t s) {
  if (!wt || !fault || !nn_conv_uses_tc(48, 16, g)) return false;
  launch_conv_tc<48, 16, true>(a4, s1, wt, bias, g, relu, out_bf, nullptr, 0, fault, s);
  return true;
}

void nn_conv_wgrad(const bf16* in, int cin, const bf16* dout, int cout, NNGrid g, float* gw,
                   float* gb, cudaStream_t s) {
  const int M = g.D * g.H * g.W;
  const int chunk = 1024;
  const int parts = (M + chunk - 1) / chunk;
  const int warps = 27 * parts;
  const int blocks = (warps + 3) / 4;
  if (cin == 16 && cout == 16) conv_wgrad_kernel<16, 16><<<blocks, 128, 0, s>>>(in, dout, g, chunk, gw);
  else if (cin == 16 && cout == 32) conv_wgrad_kernel<16, 32><<<blocks, 128, 0, s>>>(in, dout, g, chunk, gw);
  else if (cin == 32 && cout == 32) conv_wgrad_kernel<32, 32><<<blocks, 128, 0, s>>>(in, dout, g, chunk, gw);
  else if (cin == 48 && cout == 16) conv_wgrad_kernel<48, 16><<<blocks, 128, 0, s>>>(in, dout, g, chunk, gw);
  const int bchunk = 256, bparts = (M + bchunk - 1) / bchunk;
  const int per_block = 256 / cout;
  bias_grad_kernel<<<(bparts + per_block - 1) / per_block, 256, 0, s>>>(dout, M, cout, bchunk, gb);
}

void nn_pool2(const bf16* in, NNGrid f, int C, bf16* out, cudaStream_t s) {
  pool2_kernel<<<grid1((long long)f.D * f.H * f.W * C / 64, 256), 256, 0, s>>>(in, f, C, out);
}
void nn_upcat(const bf16* a4, const bf16* s1, NNGrid f, bf16* cat, cudaStream_t s) {
  upcat_kernel<<<grid1((long long)f.D * f.H * f.W * 6, 256), 256, 0, s>>>(a4, s1, f, cat);
}
void nn_mask(const float* d, const bf16* act, long long n, bf16* out, cudaStream_t s) {
  mask_kernel<<<grid1(n, 256), 256, 0, s>>>(d, act, n, out);
}
void nn_up_grad(const float* dcat, const bf16* a4, NNGrid f, bf16* out, cudaStream_t s) {
  up_grad_kernel<<<grid1((long long)f.D * f.H * f.W * 4, 256), 256, 0, s>>>(dcat, a4, f, out);
}
void nn_skip_grad(const float* dcat, const float* dp, const bf16* s1, NNGrid f, bf16* out, cudaStream_t s) {
  skip_grad_kernel<<<grid1((long long)f.D * f.H * f.W * 16, 256), 256, 0, s>>>(dcat, dp, s1, f, out);
}
void nn_mse(const float* y, const float* tgt, int M, bf16* dy, float* loss, cudaStream_t s) {
  mse_kernel<<<grid1(M, 256), 256, 0, s>>>(y, tgt, M, dy, loss);
}
void nn_adam(float* p, float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<grid1(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, c1, c2, 1e-8f);
}
void nn_pack(const float* w, int cin, int cout, bf16* wk, bf16* wb, bf16* wkt, bf16* wbt, cudaStream_t s) {
  pack_kernel<<<grid1(27 * cin * cout, 256), 256, 0, s>>>(w, cin, cout, wk, wb, wkt, wbt);
}

}  // namespace fx

// ======================================================================================
// Host side: the network object (weights, Adam state, activations for one grid,
// snapshot store) and its C ABI.
// ======================================================================================

namespace fx {
namespace {

constexpr int kLayers = 6;
constexpr int kCin[kLayers] = {16, 16, 16, 32, 48, 16};
constexpr int kCout[kLayers] = {16, 16, 32, 32, 16, 16};

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, long long n, bf16* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = __float2bfloat16(in[t]);
}


}  // namespace
}  // namespace fx

using fx::bf16;

struct ferrox_nn {
  fx::NNGrid g{}, gc{};
  int M = 0, Mc = 0;
  cudaStream_t stream = nullptr;
  float* w[fx::kLayers] = {};
  float* b[fx::kLayers] = {};
  float* gw[fx::kLayers] = {};
  float* gb[fx::kLayers] = {};
  float* mw[fx::kLayers] = {};
  float* vw[fx::kLayers] = {};
  float* mb[fx::kLayers] = {};
  float* vb[fx::kLayers] = {};
  bf16* wk[fx::kLayers] = {};
  bf16* wb[fx::kLayers] = {};
  bf16* wkt[fx::kLayers] = {};   // tensor-memory operand layouts of wk and wb
  bf16* wbt[fx::kLayers] = {};
  int* fault = nullptr;          // set by a tensor-memory convolution whose wait ran out
  bool tc = true;                // tensor-memory convolutions where the grid allows
  bf16 *x = nullptr, *a1 = nullptr, *s1 = nullptr, *p = nullptr, *a3 = nullptr, *a4 = nullptr,
       *cat = nullptr, *a5 = nullptr, *dy = nullptr, *t16a = nullptr, *t16b = nullptr,
       *t32a = nullptr, *t32b = nullptr, *tcoarse16 = nullptr;
  float *y = nullptr, *df = nullptr, *dcat = nullptr, *dpc = nullptr, *loss = nullptr;
  int cap = 0, count = 0, next = 0;
  bf16* snap_x = nullptr;     // [cap][M][16]
  float* snap_t = nullptr;    // [cap][M]
  int adam_step = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

std::string g_nn_error;

ferrox_status nfail(ferrox_nn* n, ferrox_status s, const std::string& m) {
  if (n) n->err = m; else g_nn_error = m;
  return s;
}

#define FX_NCK(call)                                                                          \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return nfail(N, _e == cudaErrorMemoryAllocation ? FERROX_ENOMEM : FERROX_ECUDA,         \
                   std::string(#call) + ": " + cudaGetErrorString(_e));                       \
  } while (0)

template <typename P>
cudaError_t nalloc(ferrox_nn* N, P** ptr, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e == cudaSuccess) {
    N->allocs.push_back(v);
    cudaMemset(v, 0, bytes);
  }
  *ptr = static_cast<P*>(v);
  return e;
}

void repack(ferrox_nn* N) {
  for (int l = 0; l < fx::kLayers; ++l)
    fx::nn_pack(N->w[l], fx::kCin[l], fx::kCout[l], N->wk[l], N->wb[l], N->wkt[l], N->wbt[l], N->stream);
}

// one convolution of layer l: forward weights, or the adjoint's when adjoint is set
void conv(ferrox_nn* N, int l, bool adjoint, const bf16* in, fx::NNGrid g, int relu, bf16* out_bf, float* out_f,
          cudaStream_t s, int f_ch0 = 0) {
  const int cin = adjoint ? fx::kCout[l] : fx::kCin[l], cout = adjoint ? fx::kCin[l] : fx::kCout[l];
  fx::nn_conv_fwd(in, cin, adjoint ? N->wb[l] : N->wk[l], !N->tc ? nullptr : adjoint ? N->wbt[l] : N->wkt[l],
                  adjoint ? nullptr : N->b[l], cout, g, relu, out_bf, out_f, f_ch0, N->fault, s);
}

// forward pass from N->x; output channel 0 (FP32) in N->y.  The concatenation
// [up(a4), s1] is formed in memory only for a backward pass (keep_cat) or where
// the tensor-memory kernel cannot read it in place.
void forward(ferrox_nn* N, bool keep_cat) {
  cudaStream_t s = N->stream;
  using namespace fx;
  conv(N, 0, false, N->x, N->g, 1, N->a1, nullptr, s);
  conv(N, 1, false, N->a1, N->g, 1, N->s1, nullptr, s);
  nn_pool2(N->s1, N->g, 16, N->p, s);
  conv(N, 2, false, N->p, N->gc, 1, N->a3, nullptr, s);
  conv(N, 3, false, N->a3, N->gc, 1, N->a4, nullptr, s);
  if (keep_cat || !N->tc ||
      !nn_conv_upcat_tc(N->a4, N->s1, N->wkt[4], N->b[4], N->g, 1, N->a5, N->fault, s)) {
    nn_upcat(N->a4, N->s1, N->g, N->cat, s);
    conv(N, 4, false, N->cat, N->g, 1, N->a5, nullptr, s);
  }
  conv(N, 5, false, N->a5, N->g, 0, nullptr, N->y, s, 1);   // output channel 0 only
}

// backward pass from N->dy (gradient of the loss w.r.t. the output); accumulates gw, gb
void backward(ferrox_nn* N) {
  cudaStream_t s = N->stream;
  using namespace fx;
  const long long M = N->M, Mc = N->Mc;
  nn_conv_wgrad(N->a5, 16, N->dy, 16, N->g, N->gw[5], N->gb[5], s);
  conv(N, 5, true, N->dy, N->g, 0, nullptr, N->df, s);
  nn_mask(N->df, N->a5, M * 16, N->t16a, s);                                  // da5
  nn_conv_wgrad(N->cat, 48, N->t16a, 16, N->g, N->gw[4], N->gb[4], s);
  conv(N, 4, true, N->t16a, N->g, 0, nullptr, N->dcat, s);
  nn_up_grad(N->dcat, N->a4, N->g, N->t32a, s);                               // da4
  nn_conv_wgrad(N->a3, 32, N->t32a, 32, N->gc, N->gw[3], N->gb[3], s);
  conv(N, 3, true, N->t32a, N->gc, 0, nullptr, N->df, s);
  nn_mask(N->df, N->a3, Mc * 32, N->t32b, s);                                 // da3
  nn_conv_wgrad(N->p, 16, N->t32b, 32, N->gc, N->gw[2], N->gb[2], s);
  conv(N, 2, true, N->t32b, N->gc, 0, nullptr, N->dpc, s);                   // dp
  nn_skip_grad(N->dcat, N->dpc, N->s1, N->g, N->t16b, s);                     // ds1
  nn_conv_wgrad(N->a1, 16, N->t16b, 16, N->g, N->gw[1], N->gb[1], s);
  conv(N, 1, true, N->t16b, N->g, 0, nullptr, N->df, s);
  nn_mask(N->df, N->a1, M * 16, N->t16a, s);                                  // da1
  nn_conv_wgrad(N->x, 16, N->t16a, 16, N->g, N->gw[0], N->gb[0], s);
}

void nn_release(ferrox_nn* N) {
  if (!N) return;
  if (N->stream) cudaStreamSynchronize(N->stream);
  for (void* p : N->allocs) cudaFree(p);
  delete N;
}

}  // namespace

namespace fx {
// used by the context when it feeds the network (engine.cu)
bf16* nn_input(ferrox_nn* N) { return N->x; }
const float* nn_output(ferrox_nn* N) { return N->y; }
void nn_run_forward(ferrox_nn* N, cudaStream_t s) {
  cudaStream_t keep = N->stream;
  N->stream = s;
  forward(N, false);
  N->stream = keep;
}
NNGrid nn_grid(const ferrox_nn* N) { return N->g; }
int nn_capacity(const ferrox_nn* N) { return N->cap; }
bf16* nn_snap_x(ferrox_nn* N) { return N->snap_x; }
float* nn_snap_t(ferrox_nn* N) { return N->snap_t; }
int nn_next_slot(const ferrox_nn* N) { return N->next; }
void nn_note_snapshots(ferrox_nn* N, int added) {
  N->count = std::min(N->cap, N->count + added);
  N->next = (N->next + added) % std::max(1, N->cap);
}
}  // namespace fx

extern "C" {

ferrox_status ferrox_nn_create(ferrox_nn** out, int D, int H, int W, int capacity,
                               const float* weights, const float* biases, void* cuda_stream) {
  if (!out) return nfail(nullptr, FERROX_EINVAL, "null output pointer");
  *out = nullptr;
  if (D < 2 || H < 2 || W < 2 || D % 2 || H % 2 || W % 2)
    return nfail(nullptr, FERROX_EINVAL, "network grid sizes must be even and >= 2");
  if (capacity < 0 || !weights || !biases) return nfail(nullptr, FERROX_EINVAL, "bad argument");
  ferrox_nn* N = new ferrox_nn();
  N->g = fx::NNGrid{D, H, W};
  N->gc = fx::NNGrid{D / 2, H / 2, W / 2};
  N->M = D * H * W;
  N->Mc = N->M / 8;
  N->cap = capacity;
  N->stream = static_cast<cudaStream_t>(cuda_stream);
  if (const cudaError_t te = fx::nn_tc_setup(); te != cudaSuccess) {
    delete N;
    return nfail(nullptr, FERROX_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(te));
  }
  const size_t M = N->M, Mc = N->Mc;
  auto fail_alloc = [&](cudaError_t e) {
    const std::string m = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    nn_release(N);
    return nfail(nullptr, FERROX_ENOMEM, m);
  };
  cudaError_t e;
  size_t woff = 0, boff = 0;
  for (int l = 0; l < fx::kLayers; ++l) {
    const size_t nw = 27 * fx::kCin[l] * fx::kCout[l], nb = fx::kCout[l];
    for (float** p : {&N->w[l], &N->gw[l], &N->mw[l], &N->vw[l]})
      if ((e = nalloc(N, p, nw * sizeof(float))) != cudaSuccess) return fail_alloc(e);
    for (float** p : {&N->b[l], &N->gb[l], &N->mb[l], &N->vb[l]})
      if ((e = nalloc(N, p, nb * sizeof(float))) != cudaSuccess) return fail_alloc(e);
    if ((e = nalloc(N, &N->wk[l], nw * sizeof(bf16))) != cudaSuccess) return fail_alloc(e);
    if ((e = nalloc(N, &N->wb[l], nw * sizeof(bf16))) != cudaSuccess) return fail_alloc(e);
    if ((e = nalloc(N, &N->wkt[l], nw * sizeof(bf16))) != cudaSuccess) return fail_alloc(e);
    if ((e = nalloc(N, &N->wbt[l], nw * sizeof(bf16))) != cudaSuccess) return fail_alloc(e);
    cudaMemcpy(N->w[l], weights + woff, nw * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(N->b[l], biases + boff, nb * sizeof(float), cudaMemcpyHostToDevice);
    woff += nw;
    boff += nb;
  }
  struct { bf16** p; size_t n; } bufs[] = {
      {&N->x, M * 16}, {&N->a1, M * 16}, {&N->s1, M * 16}, {&N->p, Mc * 16}, {&N->a3, Mc * 32},
      {&N->a4, Mc * 32}, {&N->cat, M * 48}, {&N->a5, M * 16}, {&N->dy, M * 16},
      {&N->t16a, M * 16}, {&N->t16b, M * 16}, {&N->t32a, Mc * 32}, {&N->t32b, Mc * 32},
      {&N->tcoarse16, Mc * 16}};
  for (auto& bq : bufs)
    if ((e = nalloc(N, bq.p, bq.n * sizeof(bf16))) != cudaSuccess) return fail_alloc(e);
  struct { float** p; size_t n; } fbufs[] = {{&N->y, M}, {&N->df, M * 48}, {&N->dcat, M * 48},
                                              {&N->dpc, Mc * 16}, {&N->loss, 4}};
  for (auto& bq : fbufs)
    if ((e = nalloc(N, bq.p, bq.n * sizeof(float))) != cudaSuccess) return fail_alloc(e);
  if ((e = nalloc(N, &N->fault, sizeof(int))) != cudaSuccess) return fail_alloc(e);
  if (capacity > 0) {
    if ((e = nalloc(N, &N->snap_x, (size_t)capacity * M * 16 * sizeof(bf16))) != cudaSuccess) return fail_alloc(e);
    if ((e = nalloc(N, &N->snap_t, (size_t)capacity * M * sizeof(float))) != cudaSuccess) return fail_alloc(e);
  }
  repack(N);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    nn_release(N);
    return nfail(nullptr, FERROX_ECUDA, cudaGetErrorString(e));
  }
  *out = N;
  return FERROX_OK;
}

ferrox_status ferrox_nn_forward(ferrox_nn* N, const float* x_dev, float* y_dev) {
  if (!N || !x_dev || !y_dev) return nfail(N, FERROX_EINVAL, "null argument");
  fx::f32_to_bf16_kernel<<<fx::grid1((long long)N->M * 16, 256), 256, 0, N->stream>>>(x_dev, (long long)N->M * 16, N->x);
  forward(N, false);
  FX_NCK(cudaMemcpyAsync(y_dev, N->y, (size_t)N->M * sizeof(float), cudaMemcpyDeviceToDevice, N->stream));
  FX_NCK(cudaGetLastError());
  return FERROX_OK;
}

// forward + MSE against t_dev + backward: gradients are accumulated (not applied)
ferrox_status ferrox_nn_loss_grad(ferrox_nn* N, const float* x_dev, const float* t_dev, float* loss_host) {
  if (!N || !x_dev || !t_dev) return nfail(N, FERROX_EINVAL, "null argument");
  fx::f32_to_bf16_kernel<<<fx::grid1((long long)N->M * 16, 256), 256, 0, N->stream>>>(x_dev, (long long)N->M * 16, N->x);
  FX_NCK(cudaMemsetAsync(N->loss, 0, sizeof(float), N->stream));
  forward(N, true);
  fx::nn_mse(N->y, t_dev, N->M, N->dy, N->loss, N->stream);
  backward(N);
  FX_NCK(cudaGetLastError());
  if (loss_host) {
    FX_NCK(cudaMemcpyAsync(loss_host, N->loss, sizeof(float), cudaMemcpyDeviceToHost, N->stream));
    FX_NCK(cudaStreamSynchronize(N->stream));
  }
  return FERROX_OK;
}

ferrox_status ferrox_nn_params(ferrox_nn* N, float* w, float* b, float* gw, float* gb) {
  if (!N) return nfail(nullptr, FERROX_EINVAL, "null network");
  FX_NCK(cudaStreamSynchronize(N->stream));
  size_t woff = 0, boff = 0;
  for (int l = 0; l < fx::kLayers; ++l) {
    const size_t nw = 27 * fx::kCin[l] * fx::kCout[l], nb = fx::kCout[l];
    if (w) FX_NCK(cudaMemcpy(w + woff, N->w[l], nw * sizeof(float), cudaMemcpyDeviceToHost));
    if (b) FX_NCK(cudaMemcpy(b + boff, N->b[l], nb * sizeof(float), cudaMemcpyDeviceToHost));
    if (gw) FX_NCK(cudaMemcpy(gw + woff, N->gw[l], nw * sizeof(float), cudaMemcpyDeviceToHost));
    if (gb) FX_NCK(cudaMemcpy(gb + boff, N->gb[l], nb * sizeof(float), cudaMemcpyDeviceToHost));
    woff += nw;
    boff += nb;
  }
  return FERROX_OK;
}

ferrox_status ferrox_nn_set_params(ferrox_nn* N, const float* w, const float* b) {
  if (!N || !w || !b) return nfail(N, FERROX_EINVAL, "null argument");
  size_t woff = 0, boff = 0;
  for (int l = 0; l < fx::kLayers; ++l) {
    const size_t nw = 27 * fx::kCin[l] * fx::kCout[l], nb = fx::kCout[l];
    FX_NCK(cudaMemcpyAsync(N->w[l], w + woff, nw * sizeof(float), cudaMemcpyHostToDevice, N->stream));
    FX_NCK(cudaMemcpyAsync(N->b[l], b + boff, nb * sizeof(float), cudaMemcpyHostToDevice, N->stream));
    woff += nw;
    boff += nb;
  }
  repack(N);
  FX_NCK(cudaStreamSynchronize(N->stream));
  return FERROX_OK;
}

ferrox_status ferrox_nn_adam_step(ferrox_nn* N, double lr) {
  if (!N || !(lr > 0.0)) return nfail(N, FERROX_EINVAL, "bad argument");
  N->adam_step += 1;
  for (int l = 0; l < fx::kLayers; ++l) {
    const int nw = 27 * fx::kCin[l] * fx::kCout[l], nb = fx::kCout[l];
    fx::nn_adam(N->w[l], N->gw[l], N->mw[l], N->vw[l], nw, (float)lr, N->adam_step, N->stream);
    fx::nn_adam(N->b[l], N->gb[l], N->mb[l], N->vb[l], nb, (float)lr, N->adam_step, N->stream);
  }
  repack(N);
  FX_NCK(cudaGetLastError());
  return FERROX_OK;
}

ferrox_status ferrox_nn_snapshot_count(const ferrox_nn* N, int* count) {
  if (!N || !count) return FERROX_EINVAL;
  *count = N->count;
  return FERROX_OK;
}

// epochs over the stored snapshots (in storage order), Adam every `batch`
// snapshots; loss_per_epoch[e] = mean snapshot loss of epoch e
ferrox_status ferrox_nn_train(ferrox_nn* N, int epochs, double lr, int batch, float* loss_per_epoch) {
  if (!N || epochs < 0 || batch < 1 || !(lr > 0.0)) return nfail(N, FERROX_EINVAL, "bad argument");
  if (N->count < 1) return nfail(N, FERROX_ESTATE, "no snapshots collected");
  const size_t M = N->M;
  // a fresh order of the snapshots every epoch (Fisher-Yates with a splitmix64
  // stream of fixed seed, so runs repeat), and a cosine decay of the step size
  // from lr to lr / 10 over all Adam steps of the call
  std::vector<int> order(N->count);
  for (int q = 0; q < N->count; ++q) order[q] = q;
  unsigned long long state = 0x2545F4914F6CDD1Dull;
  auto next = [&state]() {
    unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const long long per_epoch = (N->count + batch - 1) / batch, total = std::max(1LL, per_epoch * epochs);
  long long k = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int q = N->count - 1; q > 0; --q) std::swap(order[q], order[(int)(next() % (unsigned long long)(q + 1))]);
    FX_NCK(cudaMemsetAsync(N->loss, 0, sizeof(float), N->stream));
    for (int j = 0; j < N->count; ++j) {
      const int q = order[j];
      FX_NCK(cudaMemcpyAsync(N->x, N->snap_x + (size_t)q * M * 16, M * 16 * sizeof(bf16),
                             cudaMemcpyDeviceToDevice, N->stream));
      forward(N, true);
      fx::nn_mse(N->y, N->snap_t + (size_t)q * M, N->M, N->dy, N->loss, N->stream);
      backward(N);
      if ((j + 1) % batch == 0 || j + 1 == N->count) {
        const double lr_k = lr * (0.1 + 0.45 * (1.0 + std::cos(3.141592653589793 * (double)k / (double)total)));
        ++k;
        N->adam_step += 1;
        for (int l = 0; l < fx::kLayers; ++l) {
          const int nw = 27 * fx::kCin[l] * fx::kCout[l], nb = fx::kCout[l];
          fx::nn_adam(N->w[l], N->gw[l], N->mw[l], N->vw[l], nw, (float)lr_k, N->adam_step, N->stream);
          fx::nn_adam(N->b[l], N->gb[l], N->mb[l], N->vb[l], nb, (float)lr_k, N->adam_step, N->stream);
        }
        repack(N);
      }
    }
    FX_NCK(cudaGetLastError());
    float l = 0.f;
    FX_NCK(cudaMemcpyAsync(&l, N->loss, sizeof(float), cudaMemcpyDeviceToHost, N->stream));
    FX_NCK(cudaStreamSynchronize(N->stream));
    if (loss_per_epoch) loss_per_epoch[ep] = l / N->count;
  }
  return FERROX_OK;
}

ferrox_status ferrox_nn_destroy(ferrox_nn* N) {
  nn_release(N);
  return FERROX_OK;
}

const char* ferrox_nn_last_error(const ferrox_nn* N) { return N ? N->err.c_str() : g_nn_error.c_str(); }

ferrox_status ferrox_nn_use_tensor_memory(ferrox_nn* N, int on) {
  if (!N || (on != 0 && on != 1)) return nfail(N, FERROX_EINVAL, "use_tensor_memory must be 0 or 1");
  N->tc = on != 0;
  return FERROX_OK;
}

ferrox_status ferrox_nn_kernel_info(ferrox_nn* N, int* tc_forward, int* tc_backward, int* fault) {
  if (!N) return nfail(nullptr, FERROX_EINVAL, "null network");
  int f = 0, b = 0;
  if (N->tc) {
    for (int l = 0; l < fx::kLayers; ++l) {
      const fx::NNGrid g = (l == 2 || l == 3) ? N->gc : N->g;
      f += fx::nn_conv_uses_tc(fx::kCin[l], fx::kCout[l], g);
      if (l > 0) b += fx::nn_conv_uses_tc(fx::kCout[l], fx::kCin[l], g);
    }
  }
  if (tc_forward) *tc_forward = f;
  if (tc_backward) *tc_backward = b;
  if (fault) {
    FX_NCK(cudaStreamSynchronize(N->stream));
    FX_NCK(cudaMemcpy(fault, N->fault, sizeof(int), cudaMemcpyDeviceToHost));
  }
  return FERROX_OK;
}

}  // extern "C"

// ======================================================================================
// Bridge between the multigrid arenas and the network (used by the context).
// ======================================================================================
namespace fx {
namespace {

// 2x2x2 (or semi-coarsened) mean of a level field into the next level
template <typename T>
__global__ void avg_down_kernel(T* __restrict__ a, LevelDesc F, LevelDesc C) {
  const long long n = C.ncell;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % C.nx), J = (int)((t / C.nx) % C.ny), K = (int)(t / ((long long)C.nx * C.ny));
    const int nxc = F.crx ? 2 : 1, nyc = F.cry ? 2 : 1, nzc = F.crz ? 2 : 1;
    double s = 0.0;
    for (int dk = 0; dk < nzc; ++dk)
      for (int dj = 0; dj < nyc; ++dj)
        for (int di = 0; di < nxc; ++di) {
          const int i = F.crx ? 2 * I + di : I, j = F.cry ? 2 * J + dj : J, k = F.crz ? 2 * K + dk : K;
          s += (double)a[F.off + ((long long)k * F.ny + j) * F.nx + i];
        }
    a[C.off + t] = (T)(s / (nxc * nyc * nzc));
  }
}

// sum of squares of a level field in fixed order: one block
template <typename T>
__global__ void rms_kernel(const T* __restrict__ a, long long off, long long n, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) {
    const double v = (double)a[off + t];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = sqrt(s / (double)n) + 1e-300;
  }
}

// network input: residual / rms, per-plane material features, height, bias
template <typename T>
__global__ void features_kernel(const T* __restrict__ r, LevelDesc L, const float* __restrict__ pf,
                                const double* __restrict__ scale, const DevParams* __restrict__ prm,
                                bf16* __restrict__ x) {
  const long long n = L.ncell;
  const float inv = (float)(1.0 / *scale);
  const float vapp = (float)(prm->v_top - prm->v_bot);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int K = (int)(t / ((long long)L.nx * L.ny));
    float f[16] = {(float)r[L.off + t] * inv, pf[4 * K], pf[4 * K + 1], pf[4 * K + 2], pf[4 * K + 3],
                   0.5f * vapp, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(x + t * 16);
#pragma unroll
    for (int c = 0; c < 8; ++c) o[c] = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
  }
}

// e (level) = scale * network output channel 0
template <typename T>
__global__ void apply_kernel(const float* __restrict__ y, LevelDesc L, const double* __restrict__ scale,
                             T* __restrict__ e) {
  const double s = *scale;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L.ncell; t += (long long)gridDim.x * blockDim.x)
    e[L.off + t] = (T)(s * (double)y[t]);
}

// e0 = phi - phi_guess (fine level), the error the initial guess had
template <typename T>
__global__ void guess_error_kernel(const double* __restrict__ phi, const double* __restrict__ guess,
                                   long long n, T* __restrict__ e0) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    e0[t] = (T)(phi[t] - guess[t]);
}

// training target = restricted error / rms of the restricted initial residual
template <typename T>
__global__ void target_kernel(const T* __restrict__ e, LevelDesc L, const double* __restrict__ scale,
                              float* __restrict__ tgt) {
  const double inv = 1.0 / *scale;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L.ncell; t += (long long)gridDim.x * blockDim.x)
    tgt[t] = (float)((double)e[L.off + t] * inv);
}

}  // namespace

template <typename T>
void nn_bridge_restrict(T* arena, const std::vector<LevelDesc>& lv, int to, cudaStream_t s) {
  for (int l = 0; l < to; ++l)
    avg_down_kernel<T><<<grid1(lv[l + 1].ncell, 256), 256, 0, s>>>(arena, lv[l], lv[l + 1]);
}
template <typename T>
void nn_bridge_scale(const T* arena, const LevelDesc& L, double* scale, cudaStream_t s) {
  rms_kernel<T><<<1, 1024, 0, s>>>(arena, L.off, L.ncell, scale);
}
template <typename T>
void nn_bridge_features(const T* r, const LevelDesc& L, const float* pf, const double* scale,
                        const DevParams* prm, bf16* x, cudaStream_t s) {
  features_kernel<T><<<grid1(L.ncell, 256), 256, 0, s>>>(r, L, pf, scale, prm, x);
}
template <typename T>
void nn_bridge_apply(const float* y, const LevelDesc& L, const double* scale, T* e, cudaStream_t s) {
  apply_kernel<T><<<grid1(L.ncell, 256), 256, 0, s>>>(y, L, scale, e);
}
template <typename T>
void nn_bridge_guess_error(const double* phi, const double* guess, long long n, T* e0, cudaStream_t s) {
  guess_error_kernel<T><<<grid1(n, 256), 256, 0, s>>>(phi, guess, n, e0);
}
template <typename T>
void nn_bridge_target(const T* e, const LevelDesc& L, const double* scale, float* tgt, cudaStream_t s) {
  target_kernel<T><<<grid1(L.ncell, 256), 256, 0, s>>>(e, L, scale, tgt);
}

#define FX_NNB(T)                                                                                   \
  template void nn_bridge_restrict<T>(T*, const std::vector<LevelDesc>&, int, cudaStream_t);        \
  template void nn_bridge_scale<T>(const T*, const LevelDesc&, double*, cudaStream_t);              \
  template void nn_bridge_features<T>(const T*, const LevelDesc&, const float*, const double*,      \
                                      const DevParams*, bf16*, cudaStream_t);                       \
  template void nn_bridge_apply<T>(const float*, const LevelDesc&, const double*, T*, cudaStream_t); \
  template void nn_bridge_guess_error<T>(const double*, const double*, long long, T*, cudaStream_t); \
  template void nn_bridge_target<T>(const T*, const LevelDesc&, const double*, float*, cudaStream_t);
FX_NNB(float)
FX_NNB(double)
#undef FX_NNB

}  // namespace fx
