// Capacitance C = sum_i Yh_i^T Yh_i and B y (the Gram form of Eq. 12's
// capacitance and the Woodbury right-hand side) on the 5th-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory.
//
// Per chunk of kCH = 32 tets:
//   * one producer thread stages the chunk's 112 component rows (U 54,
//     gamma 48, y 9, sqrt(w) 1) into shared memory with four 2D tensor copies
//     (TMA, one box of 32 tets x rows per array) that complete on an
//     mbarrier (two stages, the next chunk in flight);
//   * six formation warps, one tet per lane, build Yh^T = (sqrt(w) U
//     (I3 x gamma))^T, 48 rows of K = 6 x 32, in the K-major canonical layout
//     of the MMA's shared-memory operands (8-row x 16-byte core matrices),
//     and sum B y;
//   * the producer thread then issues 24 MMAs of M = 64 (rows 48..63 of A
//     lie past the tile and their results are dropped), N = 48, K = 8 (TF32
//     operands, FP32 accumulate) with A = B = the tile, and commits them to
//     an mbarrier the next chunk's formation waits on before it rewrites the
//     tile (three blocks per SM keep the tensor cores and the formation busy
//     in turn: measured faster than two tile buffers at two blocks per SM).
// At the end the 48 x 48 accumulator is read back with tcgen05.ld, made
// exactly symmetric (upper triangle mirrored) and written as this block's
// FP64 partial, like the mma.sync kernel it replaces on aligned meshes.
//
// TF32 rounding: Yh is rounded to TF32 (round to nearest) before it is
// stored, so C is the Gram matrix of the rounded rows and stays positive
// semi-definite. Tets past the end of the mesh arrive zero-filled by the
// tensor copies (w = 0), so they add nothing.
//
// Every wait is bounded (kWaitLimitNs of GPU time, kWaitSpinCap polls): on
// timeout the block raises sc->barrier_timeout, waits (bounded) for its own
// copies and MMAs in flight, frees its tensor memory and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "emu_internal.h"
#include "emu_kernels.cuh"
#include "emu_mixed.cuh"
#include "emu_syrk05.h"

namespace emu {

namespace {

constexpr int kCH = 32;                 // tets per chunk (one 128-byte box row per component)
constexpr int kRows = 54 + 48 + 9 + 1;  // component rows of a chunk
constexpr int kKC = 6 * kCH;            // K of a chunk (rows of Yh)
constexpr int kKQ = kKC / 4;            // 16-byte k-groups of a chunk
constexpr int kMA = 64;                 // M of the MMA (48 rows of Yh^T + 16 ignored rows)
// Core matrices (8 rows x 16 bytes) along K sit kLBO = 144 bytes apart, not
// 128: the 4-byte stores of a warp (32 consecutive k of one column) then
// fall into 32 different banks. 8-row groups sit kSBO apart.
constexpr int kLBO = 144;
constexpr int kSBO = kKQ * kLBO;
// The tile holds the 6 row groups of Yh^T. The MMA's A operand has M = 64:
// its groups 6 and 7 read whatever follows the tile; they only feed
// accumulator rows 48..63, which are never read.
constexpr int kTileBytes = 6 * kSBO;
// raw stage: the boxes of U (54 rows), gamma (48), y (9) and sqrt(w) (1),
// each at a 128-byte aligned offset, rows of kCH floats
constexpr int kRowBytes = kCH * 4;
constexpr int kOffG = 54 * kRowBytes, kOffY = 102 * kRowBytes, kOffW = 112 * kRowBytes;
constexpr int kStageBytes = ((kOffW + kRowBytes + 127) / 128) * 128;
constexpr unsigned kStageTx = kRows * kRowBytes;  // bytes the four copies deliver
constexpr int kStages = 2;
constexpr int kTiles = 1;  // tile buffers (one: three blocks per SM overlap formation and MMAs better than two tiles at two blocks)
// formation: thread (t, d, h) forms the 6 rows of tet t for the columns
// 16 d + 8 h .. 16 d + 8 h + 7 (a warp: 32 consecutive tets, one (d, h))
constexpr int kJ = 8;
constexpr int kFormThreads = kCH * 3 * (16 / kJ);
constexpr int kFormWarps = kFormThreads / 32;
constexpr int kThreads = kFormThreads + 32;  // + the producer warp
constexpr int kTmemCols = 64;                // accumulator: 48 of 64 allocated columns
constexpr int kLDC = kK + 1;                 // padded row of the accumulator's copy in shared memory
constexpr int kMmaPerChunk = kKC / 8;
static_assert(kCH == 32, "a warp forms 32 consecutive tets");
static_assert(kKC % 8 == 0, "K of a chunk is a multiple of the MMA's K");
static_assert(kOffG % 128 == 0 && kOffY % 128 == 0 && kOffW % 128 == 0, "boxes 128-byte aligned");

// dynamic shared memory: the tiles, the raw ring (128-byte aligned base)
constexpr size_t kSmemBytes = (size_t)kTiles * kTileBytes + (size_t)kStages * kStageBytes + 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
  unsigned long long spins = 0, t0 = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++spins;
    if ((spins & 255u) == 0u) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      if (now - t0 > limit_ns || spins > kWaitSpinCap) return false;
    }
  }
  return true;
}

// the box at (x, y) of a 2D tensor map into shared dst, completing on bar
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ---- tcgen05 ---------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between core matrices along K), stride byte offset (between 8-row
// groups along M / N), all in 16-byte units; bits 46-47 hold the descriptor
// version 1 of this architecture family.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kK >> 3) << 17) |
                            ((uint32_t)(kMA >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// the barrier completes once every MMA this thread issued so far has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's lane (32 lanes x 32 bit)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace

__global__ void __launch_bounds__(kThreads, kSyrk05BlocksPerSM)
    k_syrk05(MixArgs a, double* __restrict__ cpart, const __grid_constant__ Syrk05Maps maps) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_mma[kTiles];
  __shared__ uint32_t s_taddr;
  __shared__ int s_err;
  __shared__ float s_by[kK];
  unsigned char* base = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  unsigned char* tiles = base;
  unsigned char* stages = base + kTiles * kTileBytes;  // the raw ring
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m = a.m;
  const int64_t nch = (m + kCH - 1) / kCH;
  const int64_t G = gridDim.x;
  const int64_t nmine = (int64_t)blockIdx.x < nch ? (nch - 1 - blockIdx.x) / G + 1 : 0;
  const unsigned long long limit = kWaitLimitNs;
  const bool producer = tid == kFormThreads;  // lane 0 of the last warp

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar_full[s], 1);
    for (int t = 0; t < kTiles; ++t) mbar_init(&bar_mma[t], 1);
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&s_taddr, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;

  // producer: the four tensor copies of local chunk i into stage i % kStages
  auto issue = [&](int64_t i) {
    const int st = (int)(i % kStages);
    const int x = (int)((blockIdx.x + i * G) * kCH);  // first tet (x * 4 bytes: a multiple of 16)
    unsigned char* dst = stages + st * kStageBytes;
    fence_async_smem();  // the formation's reads of this stage came first
    mbar_expect_tx(&bar_full[st], kStageTx);
    tma_load_2d(dst, &maps.U, x, 0, &bar_full[st]);
    tma_load_2d(dst + kOffG, &maps.G, x, 0, &bar_full[st]);
    tma_load_2d(dst + kOffY, &maps.Y, x, 0, &bar_full[st]);
    tma_load_2d(dst + kOffW, &maps.W, x, 0, &bar_full[st]);
  };
  int64_t issued = 0;
  if (producer) {
    for (; issued < nmine && issued < kStages; ++issued) issue(issued);
  }

  // formation role (warps 0 .. kFormWarps - 1): tet ft, component fd, columns
  // 16 fd + 8 fh .. + 7
  const int ft = lane, fd = warp % 3, fh = warp / 3;
  float by[kJ];
#pragma unroll
  for (int jj = 0; jj < kJ; ++jj) by[jj] = 0.f;
  int64_t i = 0;
  bool err = false;
  for (; i < nmine; ++i) {
    const int st = (int)(i % kStages);
    const int tb = (int)(i % kTiles);
    bool ok = true;
    if (warp < kFormWarps) {
      ok = mbar_wait(&bar_full[st], (unsigned)((i / kStages) & 1), limit);
      // chunk i - kTiles's MMAs read this tile
      if (ok && i >= kTiles) ok = mbar_wait(&bar_mma[tb], (unsigned)((i / kTiles - 1) & 1), limit);
      if (ok) {
        const float* R = reinterpret_cast<const float*>(stages + st * kStageBytes) + ft;
        float u[6][3];
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
          for (int b = 0; b < 3; ++b) u[r][b] = R[(9 * r + 3 * fd + b) * kCH];
        const float sw = R[(kOffW / 4)];
        const float y0 = R[(102 + 3 * fd) * kCH], y1 = R[(102 + 3 * fd + 1) * kCH], y2 = R[(102 + 3 * fd + 2) * kCH];
        // k = r kCH + ft: k-group (k / 4) at kLBO, position k % 4 within the core-matrix row
        unsigned char* rowbase = tiles + tb * kTileBytes + (ft >> 2) * kLBO + (ft & 3) * 4;
#pragma unroll
        for (int jj = 0; jj < kJ; ++jj) {
          const int j = kJ * fh + jj, c = 16 * fd + j;
          const float g0 = sw * R[(54 + 3 * j) * kCH], g1 = sw * R[(54 + 3 * j + 1) * kCH],
                      g2 = sw * R[(54 + 3 * j + 2) * kCH];
          by[jj] += sw * ((g0 * y0 + g1 * y1) + g2 * y2);  // w gamma_j . y_d
          unsigned char* cb = rowbase + (c >> 3) * kSBO + (c & 7) * 16;
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            const float o = (u[r][0] * g0 + u[r][1] * g1) + u[r][2] * g2;
            *reinterpret_cast<uint32_t*>(cb + r * (kCH / 4) * kLBO) = to_tf32(o);
          }
        }
        fence_async_smem();  // the tile is read by the tensor cores next
      }
    }
    // tile i complete, stage i read; every thread learns whether any wait gave up
    if (__syncthreads_or(ok ? 0 : 1)) {
      err = true;
      break;
    }
    if (producer) {
      tc_fence_after();
      const uint32_t t0 = smem_u32(tiles + tb * kTileBytes);
#pragma unroll 1
      for (int s = 0; s < kMmaPerChunk; ++s) {
        const uint64_t d = smem_desc(t0 + 2u * kLBO * s, (uint32_t)kLBO, (uint32_t)kSBO);
        mma_tf32(taddr, d, d, (i > 0 || s > 0) ? 1u : 0u);
      }
      mma_commit(&bar_mma[tb]);
      if (issued < nmine) {  // the stage chunk i used is free: chunk i + kStages
        issue(issued);
        ++issued;
      }
    }
  }
  // drain (producer): the copies issued but not consumed (after an error) and
  // the last commit, which covers every MMA of the block
  if (producer) {
    const int64_t committed = err ? i : nmine;
    for (int64_t k = committed; k < issued; ++k)
      mbar_wait(&bar_full[k % kStages], (unsigned)((k / kStages) & 1), limit);
    if (committed > 0) {
      const int64_t k = committed - 1;
      if (!mbar_wait(&bar_mma[k % kTiles], (unsigned)((k / kTiles) & 1), limit)) atomicExch(&s_err, 1);
    }
  }
  // B y: the 32 tets of a warp summed by a fixed butterfly
  if (warp < kFormWarps) {
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) {
      float v = by[jj];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_by[16 * fd + kJ * fh + jj] = v;
    }
  }
  __syncthreads();
  const bool ok = !err && s_err == 0;
  float* sC = reinterpret_cast<float*>(tiles);  // the tiles are free once the MMAs are done
  if (ok && nmine > 0) {
    tc_fence_after();
    if (warp < 4) {
      // M = 64: accumulator rows 16 w .. 16 w + 15 sit in lanes 32 w .. 32 w + 15
      const int row = 16 * warp + lane;
#pragma unroll
      for (int cb = 0; cb < 3; ++cb) {
        uint32_t v[16];
        tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + 16u * cb, v);
        tmem_ld_wait();
        if (lane < 16 && row < kK)
#pragma unroll
          for (int t = 0; t < 16; ++t) sC[row * kLDC + 16 * cb + t] = __uint_as_float(v[t]);
      }
    }
  } else {
    for (int e = tid; e < kK * kLDC; e += kThreads) sC[e] = 0.f;
  }
  if (!ok && tid == 0) atomicExch(&a.sc->barrier_timeout, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, kTmemCols);
  }
  // this block's partials, the upper triangle mirrored (exactly symmetric)
  const size_t nb = gridDim.x;
  for (int e = tid; e < kK * kK; e += kThreads) {
    const int r = e / kK, c = e % kK;
    cpart[(size_t)e * nb + blockIdx.x] = (double)(r <= c ? sC[r * kLDC + c] : sC[c * kLDC + r]);
  }
  if (tid < kK) cpart[(size_t)(kCapEntries + tid) * nb + blockIdx.x] = ok ? (double)s_by[tid] : 0.0;
}

bool syrk05_usable(const MixArgs& a) {
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return a.m > 0 && a.m % 4 == 0 && a.sw && al16(a.Uw) && al16(a.gam) && al16(a.y) && al16(a.sw);
}

int syrk05_grid(int64_t m, int sms) {
  const int64_t nch = (m + kCH - 1) / kCH;
  const int64_t g = (int64_t)kSyrk05BlocksPerSM * sms;
  return (int)(nch < g ? (nch > 0 ? nch : 1) : g);
}

cudaError_t prepare_syrk05() {
  static bool set[64] = {false};
  static std::mutex mu;  // handles may be built from several threads
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_syrk05, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e == cudaSuccess) set[dev] = true;
  return e;
}

namespace {
// a rows x m FP32 array (row stride m) as a 2D tensor map with boxes of kCH
// tets x all rows; reads past m are zero-filled
bool encode_rows(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const float* base, int64_t m, int rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)m * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kCH, (cuuint32_t)rows};
  const cuuint32_t elem[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, elem,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

bool make_syrk05_maps(const MixArgs& a, Syrk05Maps* maps) {
  if (!syrk05_usable(a) || a.m > ((int64_t)1 << 31) - kCH) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!enc) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
              cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn)
        return false;
      enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  return encode_rows(enc, &maps->U, a.Uw, a.m, 54) && encode_rows(enc, &maps->G, a.gam, a.m, 48) &&
         encode_rows(enc, &maps->Y, a.y, a.m, 9) && encode_rows(enc, &maps->W, a.sw, a.m, 1);
}

void launch_syrk05(const MixArgs& a, const Syrk05Maps& maps, int grid, double* cpart, cudaStream_t st) {
  k_syrk05<<<grid, kThreads, kSmemBytes, st>>>(a, cpart, maps);
}

}  // namespace emu
