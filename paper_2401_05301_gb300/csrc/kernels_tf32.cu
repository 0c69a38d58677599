// Complex GEMM on the 5th-generation tensor cores as split 3xTF32 products
// with FP32 accumulation (the mixed-precision contractions: theta = B B B,
// the gate, and the rebuild of B).
//
// C (complex, FP64 in memory) = alpha * A * op(B), op(B) in {B, B^+}.
// Real embedding: A is used as stored (re/im interleaved along K, so as a real
// M x 2K matrix) and B is expanded to the real 2K x 2N matrix with 2x2 blocks
// [[br, bi], [-bi, br]]; the real product then holds (Re C, Im C) interleaved
// along its columns, i.e. exactly the complex C.
//
// Split: every FP64 operand element x is cut into tf32 hi + lo by integer
// operations on its IEEE-754 fields, both rounded to nearest, so that
// |x - hi - lo| <= 2^-23 |x| without bias.  The product keeps
// hi*hi + hi*lo + lo*hi (three MMAs per k-step) and drops lo*lo.  No FP64
// arithmetic happens in the loop: on this part FP64 runs at 1/64 of the FP32 rate.
//
// Accumulation: the tensor core's FP32 accumulation rounds towards zero, which
// over a long K becomes a bias growing linearly with K (measured -1e-4 relative
// at K = 4096 with same-sign data).  Every k-step of 8 reals therefore gets a
// fresh accumulator in tensor memory (hi*lo, lo*hi, then hi*hi: one large
// product per chain), and after each slab the threads add the four
// accumulators into FP32 registers with round-to-nearest adds (measured bias
// ~4e-8 relative, independent of K).
//
// Kernel: one CTA (256 threads) per 128 x 128 tile of the real product.
// All threads load and split a K-slab of A and B into 128-byte-swizzled,
// K-major shared-memory tiles (the canonical layout of tcgen05 matrix
// descriptors), two slabs double-buffered; one thread issues
// tcgen05.mma.kind::tf32 (M = 128, N = 128, K = 8) and commits each slab to an
// mbarrier; the next slab is loaded while the current one multiplies.  Every mbarrier
// wait is bounded (~1 s); on timeout the CTA flags an error, drains its issued
// MMAs (bounded), frees its tensor memory and returns.
#include "ptebd_internal.h"

#include <algorithm>
#include <cstdint>

namespace ptebd {

namespace {

constexpr int TM = 128;               // rows of the real product per CTA (UMMA M)
constexpr int TN = 128;               // columns of the real product per CTA (UMMA N) = 64 complex
constexpr int TK = 32;                // reals of K per slab (one 128-byte swizzle row of fp32)
constexpr int NT = 256;               // threads per CTA
constexpr int A_BYTES = TM * TK * 4;  // 16 KB per plane
constexpr int B_BYTES = TN * TK * 4;  // 16 KB per plane
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo planes of A and B: 64 KB
constexpr int NACC = TK / 8;          // one accumulator per k-step of a slab
constexpr int TMEM_COLS = NACC * TN;  // 512: the whole tensor memory of the SM
constexpr int STAGES = 2;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 128;
constexpr long long WAIT_CLOCKS = 2000000000LL;  // ~1 s at 2 GHz

// ---- small PTX wrappers ---------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CLOCKS) return false;
  }
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor for kind::tf32: D = f32, A = B = tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// x -> (hi, lo) tf32 bit patterns from the IEEE-754 fields of the double:
// hi = x rounded to 11 significant bits, lo = the remainder rounded to 11 bits.
__device__ __forceinline__ void split_tf32(double x, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t s = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  const int E = e - 1023;
  hi = 0u;
  lo = 0u;
  if (e == 0 || E < -126) return;  // zero, subnormal or below fp32 range: 0
  const long long M53 = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  long long hs = (M53 + (1ll << 41)) >> 42;  // 11-bit significand, rounded
  const long long rem = M53 - (hs << 42);    // |rem| <= 2^41
  int He = E;
  if (hs == 2048) { hs = 1024; He = E + 1; }
  if (He > 127) { hi = s | 0x7F800000u; return; }
  hi = s | ((uint32_t)(He + 127) << 23) | ((uint32_t)(hs & 0x3FF) << 13);
  if (rem == 0) return;
  const unsigned long long a = (unsigned long long)(rem < 0 ? -rem : rem);
  const int p = 63 - __clzll((long long)a);  // leading one, 0..41
  int le = E - 52 + p;
  const int sh = p - 10;
  unsigned long long ls;
  if (sh > 0) {
    ls = (a + (1ull << (sh - 1))) >> sh;
    if (ls == 2048) { ls = 1024; ++le; }
  } else {
    ls = a << (-sh);
  }
  if (le < -126) return;
  lo = (s ^ (rem < 0 ? 0x80000000u : 0u)) | ((uint32_t)(le + 127) << 23) | ((uint32_t)(ls & 0x3FF) << 13);
}

// byte offset of fp32 element (row, k) of a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t swz(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ double2 load_c(const double2* p) { return __ldg(p); }

// Fill one slab (real K offset k0) of the hi/lo planes of A and B.
__device__ void fill_slab(const TcGemmProb& P, const double2* A, const double2* B, int row0, int col0, int k0,
                          uint8_t* st) {
  uint8_t* Ahi = st;
  uint8_t* Alo = st + A_BYTES;
  uint8_t* Bhi = st + 2 * A_BYTES;
  uint8_t* Blo = st + 2 * A_BYTES + B_BYTES;
  const int kc0 = k0 >> 1;  // complex K offset of the slab
  // A: 128 rows x 16 complex; thread t handles (row = t/2, 8 complex per thread)
  for (int idx = threadIdx.x; idx < TM * 16; idx += NT) {
    const int r = idx >> 4, q = idx & 15;
    const int gr = row0 + r, gk = kc0 + q;
    double2 v = make_double2(0.0, 0.0);
    if (gr < P.M && gk < P.K) v = load_c(A + (long long)gr * P.lda + gk);
    uint32_t h0, l0, h1, l1;
    split_tf32(v.x, h0, l0);
    split_tf32(v.y, h1, l1);
    *reinterpret_cast<uint32_t*>(Ahi + swz(r, 2 * q)) = h0;
    *reinterpret_cast<uint32_t*>(Ahi + swz(r, 2 * q + 1)) = h1;
    *reinterpret_cast<uint32_t*>(Alo + swz(r, 2 * q)) = l0;
    *reinterpret_cast<uint32_t*>(Alo + swz(r, 2 * q + 1)) = l1;
  }
  // B': rows 2j, 2j+1 (j = complex column) x 32 reals of K; element b = op(B)(k, j)
  //   row 2j   : ( br, -bi ) at k' = 2k, 2k+1     row 2j+1 : ( bi, br )
  for (int idx = threadIdx.x; idx < (TN / 2) * 16; idx += NT) {
    int jj, q;
    if (P.opB == OP_N) { jj = idx & (TN / 2 - 1); q = idx / (TN / 2); } else { q = idx & 15; jj = idx >> 4; }
    const int gj = (col0 >> 1) + jj, gk = kc0 + q;
    double2 v = make_double2(0.0, 0.0);
    if (gj < P.N && gk < P.K) {
      if (P.opB == OP_N) {
        v = load_c(B + (long long)gk * P.ldb + gj);
      } else {
        v = load_c(B + (long long)gj * P.ldb + gk);
        v.y = -v.y;
      }
    }
    uint32_t hr, lr, hi_, li_;
    split_tf32(v.x, hr, lr);
    split_tf32(v.y, hi_, li_);
    const uint32_t sign = 0x80000000u;
    const int r0 = 2 * jj, r1 = 2 * jj + 1, ka = 2 * q, kb = 2 * q + 1;
    *reinterpret_cast<uint32_t*>(Bhi + swz(r0, ka)) = hr;
    *reinterpret_cast<uint32_t*>(Bhi + swz(r0, kb)) = hi_ ^ (hi_ ? sign : 0u);
    *reinterpret_cast<uint32_t*>(Bhi + swz(r1, ka)) = hi_;
    *reinterpret_cast<uint32_t*>(Bhi + swz(r1, kb)) = hr;
    *reinterpret_cast<uint32_t*>(Blo + swz(r0, ka)) = lr;
    *reinterpret_cast<uint32_t*>(Blo + swz(r0, kb)) = li_ ^ (li_ ? sign : 0u);
    *reinterpret_cast<uint32_t*>(Blo + swz(r1, ka)) = li_;
    *reinterpret_cast<uint32_t*>(Blo + swz(r1, kb)) = lr;
  }
}

// Add the 64 accumulator columns this thread owns (row 32g + lane, columns
// [64h, 64h + 64) of accumulator `which`) into acc[] with round-to-nearest adds.
__device__ __forceinline__ void drain(uint32_t tmem, int which, int g, int h, float (&acc)[64]) {
#pragma unroll
  for (int c0 = 0; c0 < 64; c0 += 16) {
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(which * TN + h * 64 + c0);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[c0 + i] = __fadd_rn(acc[c0 + i], __uint_as_float(v[i]));
  }
}

__global__ void __launch_bounds__(NT, 1) k_tf32x3(const __grid_constant__ TcGemmBatch gb) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* slab_bar = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* done_bar = slab_bar + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  int* fail_sh = reinterpret_cast<int*>(tmem_slot + 1);

  // locate the problem, batch entry and tile of this CTA
  const int tile = blockIdx.x;
  int pi = 0;
  while (pi + 1 < gb.nprob && tile >= gb.tile_start[pi + 1]) ++pi;
  const TcGemmProb& P = gb.p[pi];
  const int local = tile - gb.tile_start[pi];
  const int tn = (2 * P.N + TN - 1) / TN, tm = (P.M + TM - 1) / TM;
  const int bidx = local / (tm * tn), rr = local % (tm * tn);
  const int row0 = (rr / tn) * TM, col0 = (rr % tn) * TN;
  const double2* A = P.A + (long long)bidx * P.sA;
  const double2* B = P.B + (long long)bidx * P.sB;
  double2* C = P.C + (long long)bidx * P.sC;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp & 3, h = warp >> 2;  // TMEM lane group and column half drained by this warp
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int q = 0; q < STAGES; ++q) mbar_init(&slab_bar[q], 1);
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail_sh = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tf32_idesc(TM, TN);
  const int nk = (2 * P.K + TK - 1) / TK;  // slabs of 32 reals of K

  float acc[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) acc[i] = 0.0f;

  fill_slab(P, A, B, row0, col0, 0, smem);
  fence_async_shared();
  __syncthreads();
  bool ok = true;
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb & 1;
    if (threadIdx.x == 0) {  // slab kb: k-step kk into accumulator kk, from a fresh start
      tc_fence_after();
      uint8_t* st = smem + s * STAGE_BYTES;
      const uint32_t a_hi = smem_u32(st), a_lo = smem_u32(st + A_BYTES);
      const uint32_t b_hi = smem_u32(st + 2 * A_BYTES), b_lo = smem_u32(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
      for (int kk = 0; kk < NACC; ++kk) {
        const uint32_t off = kk * 32;  // 8 tf32 = 32 bytes along K inside the swizzled row
        const uint32_t d = tmem + (uint32_t)(kk * TN);
        mma_tf32(d, smem_desc(a_hi + off), smem_desc(b_lo + off), idesc, 0u);
        mma_tf32(d, smem_desc(a_lo + off), smem_desc(b_hi + off), idesc, 1u);
        mma_tf32(d, smem_desc(a_hi + off), smem_desc(b_hi + off), idesc, 1u);
      }
      mma_commit(&slab_bar[s]);
    }
    if (kb + 1 < nk) {  // buffer s^1 was released when slab kb-1 finished (waited below)
      fill_slab(P, A, B, row0, col0, (kb + 1) * TK, smem + (s ^ 1) * STAGE_BYTES);
      fence_async_shared();
    }
    if (mbar_wait(&slab_bar[s], (uint32_t)((kb >> 1) & 1))) {
#pragma unroll
      for (int q = 0; q < NACC; ++q) drain(tmem, q, g, h, acc);
    } else {
      atomicExch(fail_sh, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (*fail_sh) { ok = false; break; }
  }
  if (!ok) {  // let every issued MMA finish (bounded) before the tensor memory is freed
    if (threadIdx.x == 0) mma_commit(done_bar);
    mbar_wait(done_bar, 0);
  }
  tc_fence_before();
  if (ok) {
    const int row = row0 + 32 * g + lane;
    if (row < P.M) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = (col0 + h * 64) / 2 + i;
        if (j < P.N)
          C[(long long)row * P.ldc + j] =
              make_double2((double)acc[2 * i] * P.alpha, (double)acc[2 * i + 1] * P.alpha);
      }
    }
  } else if (threadIdx.x == 0 && gb.status) {
    atomicExch(gb.status, -6);  // TEBD_ERR_TIMEOUT: a bounded mbarrier wait ran out
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace

static_assert(sizeof(TcGemmBatch) < 4000, "kernel parameter block too large");
static_assert(tf32_idesc(128, 128) == ((1u << 4) | (2u << 7) | (2u << 10) | (16u << 17) | (8u << 24)), "idesc");

int tc_gemm_launch(const std::vector<TcGemmProb>& probs, int* status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  int launches = 0;
  size_t i = 0;
  while (i < probs.size()) {
    TcGemmBatch gb{};
    gb.status = status;
    int tiles = 0;
    while (i < probs.size() && gb.nprob < TC_MAXP) {
      const TcGemmProb& p = probs[i++];
      if (p.M <= 0 || p.N <= 0 || p.batch <= 0) continue;
      gb.p[gb.nprob] = p;
      gb.tile_start[gb.nprob] = tiles;
      tiles += p.batch * ((p.M + TM - 1) / TM) * ((2 * p.N + TN - 1) / TN);
      gb.nprob++;
    }
    gb.tile_start[gb.nprob] = tiles;
    if (tiles == 0) continue;
    k_tf32x3<<<tiles, NT, SMEM_BYTES, s>>>(gb);
    ++launches;
  }
  return launches;
}

}  // namespace ptebd
