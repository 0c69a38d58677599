// FP64-accurate complex GEMM on the bf16 tensor cores by exact digit splitting
// (the Ozaki scheme), for the dense products of the truncated SVD (Sec. II B) in
// the tensor-core paths: the Gram matrices H = theta' theta'^+, the projections
// Y = U^+ theta', the Hermitian rank-64 updates of the blocked reduction, the
// blocks of the back-transformation and the Newton-Schulz products (real
// operands, real results); with precision 2 also the contractions of theta and
// the rebuilds.
//
// Representation.  Every operand row is given an exponent e (|x| < 2^e over the
// row) and each real x of it becomes the integer F = round(x 2^(56-e)),
// |F| < 2^56, cut into eight balanced base-128 digits
//     F = sum_s d_s 128^(7-s),   |d_0| <= 128,  |d_s| <= 64 (s >= 1),
// each exact in bf16.  So x = 2^(e-7) sum_s d_s 2^(-7s), to 2^-56 of the row's
// largest element (the same form as an FP64 rounding bound, eight times smaller).
//
// Product.  a.b = 2^(e_a + e_b - 14) sum_{s,t} d_s(a) d_t(b) 2^(-7(s+t)).  Pairs
// with q = s + t share a power of two and go to one accumulator; q = 0..7 are
// kept (36 pairs), q >= 8 lie below 2^-55 |a|max |b|max and are dropped.  Over a
// chunk of 256 reals of K every partial sum of an accumulator is an integer below
// 2^24 (q = 0: 256 * 128^2 = 2^22; q >= 1: 256 (2 * 128 * 64 + (q - 1) 64^2)
// <= 10 * 2^20), so the tensor core's FP32 accumulation is exact whatever its
// rounding.  After each chunk the eight accumulators are read from tensor
// memory, converted to integers and added exactly into two 64-bit integers per
// output element:  P_hi = sum_{q<=3} I_q 2^(21-7q),  P_lo = sum_{q>=4} I_q 2^(49-7q),
// i.e. T = P_hi 2^28 + P_lo = sum_q I_q 2^(49-7q).  The whole K reduction is
// therefore exact; the only rounding is the final conversion
// a.b = (P_hi 2^28 + P_lo) 2^(e_a + e_b - 63) to FP64.  Results are bitwise
// reproducible and independent of the tile order.
//
// Complex products use the real embedding of the 3xTF32 path: a row of a is
// its interleaved (re, im) reals; a row of b is stored twice, as (br, -bi)
// ("D1", giving Re a.b) and (bi, br) ("D2", giving Im a.b).
//
// Data path.  A packing kernel writes the digits of every operand in the exact
// shared-memory image the tensor core reads (K-major, 128-byte swizzle), as 4 KB
// blocks of 32 rows x 64 reals ordered [slice][k-step][row block], so every
// tile of a slice is one contiguous bulk copy.  The GEMM kernel (one 128 x 32
// complex tile per CTA) is warp-specialised: one thread issues the bulk copies
// (the TMA engine, completion on mbarriers), one thread issues
// tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16) into eight accumulators that
// fill the 512 columns of tensor memory, and sixteen warps drain the
// accumulators into the 64-bit sums after each chunk and write the tile.  Every wait is
// bounded (~1 s): on timeout the CTA records TEBD_ERR_TIMEOUT, lets its issued
// copies and MMAs finish (bounded), frees its tensor memory and returns.
#include "ptebd_internal.h"

#include <algorithm>
#include <cstdint>

namespace ptebd {

namespace {

constexpr int OZ_S = 8;                         // digit slices
constexpr int OZ_TM = 128;                      // rows of a per tile (UMMA M)
constexpr int OZ_TNC = 32;                      // complex columns per tile
constexpr int OZ_TN = 2 * OZ_TNC;               // UMMA N: 32 rows of D1 then 32 of D2
constexpr int OZ_CHUNK = 4;                     // k-steps (of 64 reals) per exact chunk
constexpr int OZ_BLK = 4096;                    // one packed block: 32 rows x 64 bf16
constexpr int OZ_A_BYTES = 4 * OZ_BLK;          // A slice tile (128 rows)
constexpr int OZ_B_BYTES = 2 * OZ_BLK;          // B slice tile (64 rows)
constexpr int OZ_BSTAGE = OZ_S * OZ_B_BYTES;    // all slices of B for one k-step: 64 KB
constexpr int OZ_AR = 4;                        // ring of A slice tiles
constexpr int OZ_DW = 16;                       // drain warps (4 lane groups x 4 column quarters)
constexpr int OZ_NT = 32 * (OZ_DW + 2);          // + one copy warp + one MMA warp
constexpr int OZ_TMEM_COLS = 512;               // 8 accumulators x 64 columns
constexpr int OZ_BARS = 16;
constexpr int OZ_SMEM = 2 * OZ_BSTAGE + OZ_AR * OZ_A_BYTES + 1024 + OZ_BARS * 8 + 64;
constexpr int OZ_STAGE_LD = 65;                 // epilogue staging row (doubles), padded
constexpr long long OZ_WAIT = 2000000000LL;     // ~1 s at 2 GHz
constexpr int OZ_BAD = 1 << 20;                 // row exponent of a row holding NaN or Inf

static_assert(OZ_TM * OZ_STAGE_LD * 8 <= 2 * OZ_BSTAGE, "epilogue staging must fit the B stages");
static_assert(OZ_SMEM <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded parity wait; also gives up as soon as another role has flagged a failure.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (int it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (fail && *fail) return false;
      if (clock64() - t0 > OZ_WAIT) return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (TMA engine), completion counted on bar.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major, 128-byte-swizzled shared-memory matrix descriptor (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor for kind::f16: D = f32, A = B = bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// byte offset of bf16 element (row, k) in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t swz16(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + ((k & 7) << 1));
}

// The eight balanced base-128 digits of round(x 2^(56 - e)) (|x| < 2^e), taken
// from |x| with the sign applied afterwards, so that the digits of -x are exactly
// the negated digits of x (conjugate operands share digits up to sign).
__device__ __forceinline__ void oz_digits(double x, int e, int (&d)[OZ_S]) {
  long long F = 0;
  if (x != 0.0 && e != OZ_BAD) F = __double2ll_rn(ldexp(fabs(x), 56 - e));
  const int sg = (x < 0.0) ? -1 : 1;
#pragma unroll
  for (int s = OZ_S - 1; s >= 1; --s) {
    const int r = (int)((F + 64) & 127) - 64;
    d[s] = sg * r;
    F = (F - r) >> 7;
  }
  d[0] = sg * (int)F;
}

__device__ __forceinline__ uint32_t bf16_bits(int v) { return __float_as_uint((float)v) >> 16; }

// ---- packing ----------------------------------------------------------------------

// Element (r, k) of a job's operand, after the optional per-k scale and conjugation.
__device__ __forceinline__ double2 job_elem(const OzPackJob& J, int r, int k) {
  const long long at = (long long)r * J.rs + (long long)k * J.ks;
  double2 x = J.real ? make_double2(reinterpret_cast<const double*>(J.X)[at], 0.0) : J.X[at];
  if (J.scale) {
    const double f = J.scale[k / J.scale_div];
    x.x *= f;
    x.y *= f;
  }
  if (J.conj) x.y = -x.y;
  return x;
}

__device__ __forceinline__ int find_job(const OzPackBatch& pb, int blk) {
  int j = 0;
  while (j + 1 < pb.njob && blk >= pb.block_start[j + 1]) ++j;
  return j;
}

// Row exponents: one block per 32 rows of a job.
__global__ void __launch_bounds__(256) k_oz_exp(const __grid_constant__ OzPackBatch pb) {
  const int j = find_job(pb, blockIdx.x);
  const OzPackJob& J = pb.job[j];
  const int rb = blockIdx.x - pb.block_start[j];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double part[8][33];
  if (J.ks == 1) {  // rows contiguous along k: a warp per row
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = rb * 32 + warp + 8 * rr;
      double m = 0.0;
      if (r < J.rows)
        for (int k = lane; k < J.K; k += 32) {
          const double2 x = job_elem(J, r, k);
          m = fmax(m, fmax(fabs(x.x), fabs(x.y)));
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) part[0][warp + 8 * rr] = m;
    }
    __syncthreads();
  } else {  // rows contiguous across lanes: lane = row, warps split k
    const int r = rb * 32 + lane;
    double m = 0.0;
    if (r < J.rows)
      for (int k = warp; k < J.K; k += 8) {
        const double2 x = job_elem(J, r, k);
        m = fmax(m, fmax(fabs(x.x), fabs(x.y)));
      }
    part[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
      double t = part[0][lane];
      for (int w = 1; w < 8; ++w) t = fmax(t, part[w][lane]);
      part[0][lane] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    const double m = part[0][threadIdx.x];
    int e = 0;
    if (!(m <= 1.0e308)) e = OZ_BAD;  // NaN or Inf somewhere in the row
    else if (m > 0.0) frexp(m, &e);   // m < 2^e
    J.e[rb * 32 + threadIdx.x] = e;
  }
}

// Digits: one block per (row block, k-step) of a job; writes one or two planes.
__global__ void __launch_bounds__(256) k_oz_pack(const __grid_constant__ OzPackBatch pb) {
  const int j = find_job(pb, blockIdx.x);
  const OzPackJob& J = pb.job[j];
  const int local = blockIdx.x - pb.block_start[j];
  const int rb = local % J.nrb, kt = local / J.nrb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double tre[32][33], tim[32][33];
  __shared__ int esh[32];
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    int row, kk;
    if (J.ks == 1) { row = warp + 8 * rr; kk = lane; } else { row = lane; kk = warp + 8 * rr; }
    const int r = rb * 32 + row, k = kt * 32 + kk;
    double2 x = make_double2(0.0, 0.0);
    if (r < J.rows && k < J.K) x = job_elem(J, r, k);
    tre[row][kk] = x.x;
    tim[row][kk] = x.y;
  }
  if (threadIdx.x < 32) esh[threadIdx.x] = J.e[rb * 32 + threadIdx.x];
  __syncthreads();
  const size_t blk = ((size_t)kt * J.nrb + rb) * (OZ_BLK / 2);  // in bf16 elements, slice 0
  const size_t slice = (size_t)J.nkt * J.nrb * (OZ_BLK / 2);
#pragma unroll 1
  for (int rr = 0; rr < 4; ++rr) {
    const int row = warp + 8 * rr;
    const int e = esh[row];
    int dr[OZ_S], di[OZ_S];
    oz_digits(tre[row][lane], e, dr);
    oz_digits(tim[row][lane], e, di);
    const uint32_t off = swz16(row, 2 * lane) >> 1;
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
      uint16_t* P = pl ? J.P1 : J.P0;
      const int type = pl ? J.type1 : J.type0;
      if (!P) continue;
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) {
        int u, v;  // types: 0 (re, im), 1 (re, -im), 2 (im, re), 3 (-im, re)
        if (type == 0) { u = dr[s]; v = di[s]; }
        else if (type == 1) { u = dr[s]; v = -di[s]; }
        else if (type == 2) { u = di[s]; v = dr[s]; }
        else { u = -di[s]; v = dr[s]; }
        *reinterpret_cast<uint32_t*>(P + s * slice + blk + off) = bf16_bits(u) | (bf16_bits(v) << 16);
      }
    }
  }
}

// ---- the digit GEMM -----------------------------------------------------------------

__device__ __forceinline__ void tile_of(const OzTile& P, int local, int& mt, int& nt) {
  if (!P.herm) {
    mt = local / P.tiles_n;
    nt = local % P.tiles_n;
    return;
  }
  int rem = local;
  mt = 0;
  while (true) {
    const int cnt = min(P.tiles_n, (mt * OZ_TM + OZ_TM - 1) / OZ_TNC + 1);
    if (rem < cnt) break;
    rem -= cnt;
    ++mt;
  }
  nt = rem;
}

__global__ void __launch_bounds__(OZ_NT, 1) k_oz_gemm(const __grid_constant__ OzGemmBatch gb) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Bst = smem;                       // two stages of all B slices
  uint8_t* Ar = smem + 2 * OZ_BSTAGE;        // ring of A slice tiles
  uint64_t* bars = reinterpret_cast<uint64_t*>(Ar + OZ_AR * OZ_A_BYTES);
  uint64_t* fullB = bars;                    // [2]
  uint64_t* emptyB = bars + 2;               // [2]
  uint64_t* fullA = bars + 4;                // [4]
  uint64_t* emptyA = bars + 8;               // [4]
  uint64_t* accfull = bars + 12;
  uint64_t* accempty = bars + 13;
  uint64_t* done = bars + 14;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + OZ_BARS);
  volatile int* fail_sh = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tile = blockIdx.x;
  int pi = 0;
  while (pi + 1 < gb.nprob && tile >= gb.tile_start[pi + 1]) ++pi;
  const OzTile& P = gb.p[pi];
  int mt, nt;
  tile_of(P, tile - gb.tile_start[pi], mt, nt);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == OZ_DW + 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) { mbar_init(&fullB[i], 1); mbar_init(&emptyB[i], 1); }
    for (int i = 0; i < OZ_AR; ++i) { mbar_init(&fullA[i], 1); mbar_init(&emptyA[i], 1); }
    mbar_init(accfull, 1);
    mbar_init(accempty, OZ_DW);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail_sh = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nkt = P.nkt;
  const int nchunk = (nkt + OZ_CHUNK - 1) / OZ_CHUNK;
  const size_t sliceA = (size_t)nkt * P.nrbA * OZ_BLK, sliceB = (size_t)nkt * P.nrbB * OZ_BLK;

  if (warp == OZ_DW) {
    // ---- copies: per k-step all B slices (one stage), then the A slices through the ring
    if (lane == 0) {
      const uint8_t* DA = reinterpret_cast<const uint8_t*>(P.DA);
      const uint8_t* D1 = reinterpret_cast<const uint8_t*>(P.D1);
      const uint8_t* D2 = reinterpret_cast<const uint8_t*>(P.D2);
      int fA = 0, fB = 0;
      bool ok = true;
      for (int kt = 0; kt < nkt && ok; ++kt) {
        const int b = kt & 1;
        if (kt >= 2 && !mbar_wait(&emptyB[b], (uint32_t)(((kt >> 1) - 1) & 1), fail_sh)) { ok = false; break; }
        mbar_expect_tx(&fullB[b], OZ_BSTAGE);
        ++fB;
        uint8_t* dst = Bst + b * OZ_BSTAGE;
        const size_t off = ((size_t)kt * P.nrbB + nt) * OZ_BLK;
        for (int s = 0; s < OZ_S; ++s) {
          bulk_copy(dst + s * OZ_B_BYTES, D1 + s * sliceB + off, OZ_BLK, &fullB[b]);
          bulk_copy(dst + s * OZ_B_BYTES + OZ_BLK, D2 + s * sliceB + off, OZ_BLK, &fullB[b]);
        }
        const size_t offA = ((size_t)kt * P.nrbA + 4 * mt) * OZ_BLK;
        for (int s = 0; s < OZ_S; ++s, ++fA) {
          const int slot = fA & (OZ_AR - 1);
          if (fA >= OZ_AR && !mbar_wait(&emptyA[slot], (uint32_t)(((fA >> 2) - 1) & 1), fail_sh)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&fullA[slot], OZ_A_BYTES);
          bulk_copy(Ar + slot * OZ_A_BYTES, DA + s * sliceA + offA, OZ_A_BYTES, &fullA[slot]);
        }
      }
      if (!ok) {
        *fail_sh = 1;
        // let the copies already issued land before the CTA's shared memory is released
        for (int b = 0; b < 2; ++b) {  // the last fill issued into each buffer
          int last = -1;
          for (int kt = b; kt < fB; kt += 2) last = kt;
          if (last >= 0) mbar_wait(&fullB[b], (uint32_t)((last >> 1) & 1), nullptr);
        }
        for (int slot = 0; slot < OZ_AR; ++slot) {
          int last = -1;
          for (int f = slot; f < fA; f += OZ_AR) last = f;
          if (last >= 0) mbar_wait(&fullA[slot], (uint32_t)((last >> 2) & 1), nullptr);
        }
      }
    }
  } else if (warp == OZ_DW + 1) {
    // ---- MMA issue: accumulator q = s + t gets the pairs of slice s of a and slice t of b
    if (lane == 0) {
      const uint32_t idesc = bf16_idesc(OZ_TM, OZ_TN);
      int fA = 0;
      bool ok = true;
      for (int c = 0; c < nchunk && ok; ++c) {
        if (c > 0 && !mbar_wait(accempty, (uint32_t)((c - 1) & 1), fail_sh)) { ok = false; break; }
        tc_fence_after();
        const int kt0 = c * OZ_CHUNK, kt1 = min(nkt, kt0 + OZ_CHUNK);
        for (int kt = kt0; kt < kt1 && ok; ++kt) {
          const int b = kt & 1;
          if (!mbar_wait(&fullB[b], (uint32_t)((kt >> 1) & 1), fail_sh)) { ok = false; break; }
          tc_fence_after();
          const uint32_t bbase = smem_u32(Bst + b * OZ_BSTAGE);
          for (int s = 0; s < OZ_S; ++s, ++fA) {
            const int slot = fA & (OZ_AR - 1);
            if (!mbar_wait(&fullA[slot], (uint32_t)((fA >> 2) & 1), fail_sh)) { ok = false; break; }
            tc_fence_after();
            const uint32_t abase = smem_u32(Ar + slot * OZ_A_BYTES);
            for (int t = 0; t < OZ_S - s; ++t) {
              const uint32_t d = tmem + (uint32_t)((s + t) * OZ_TN);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t en = (kt == kt0 && s == 0 && kk == 0) ? 0u : 1u;
                mma_bf16(d, smem_desc(abase + kk * 32), smem_desc(bbase + t * OZ_B_BYTES + kk * 32), idesc, en);
              }
            }
            mma_commit(&emptyA[slot]);
          }
          if (ok) mma_commit(&emptyB[b]);
        }
        if (ok) mma_commit(accfull);
      }
      if (!ok) {
        *fail_sh = 1;
        mma_commit(done);  // all MMAs issued so far complete before tensor memory is freed
        mbar_wait(done, 0, nullptr);
      }
    }
  } else {
    // ---- drain: warp (g, h) owns TMEM lanes 32g.. and columns 16h.. of every accumulator
    const int g = warp & 3, h = warp >> 2;
    long long Phi[16], Plo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) { Phi[i] = 0; Plo[i] = 0; }
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
      if (!mbar_wait(accfull, (uint32_t)(c & 1), fail_sh)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) {
        const long long w = 1ll << (21 - 7 * (q & 3));
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(q * OZ_TN + 16 * h);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const long long I = (long long)__float2int_rn(__uint_as_float(v[i]));
          if (q < 4) Phi[i] += I * w;
          else Plo[i] += I * w;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty);
    }
    if (!ok) *fail_sh = 1;
    // ---- epilogue: (P_hi 2^28 + P_lo) 2^(e_a + e_b - 63), staged in shared memory.
    // Every drain warp takes the same branch: the decision is an OR over their own
    // outcomes, reduced by the named barrier itself (all chunks drained => all MMAs done).
    int any_bad;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(any_bad)
        : "r"(ok ? 0 : 1), "r"(32 * OZ_DW)
        : "memory");
    if (!any_bad) {
      double* stage = reinterpret_cast<double*>(Bst);
      const int il = 32 * g + lane, row = mt * OZ_TM + il;
      const int ea = (row < P.M) ? P.eA[row] : 0;
      const int c0 = 16 * h;  // first staged column (0..31: D1 -> Re, 32..63: D2 -> Im)
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = nt * OZ_TNC + ((c0 + i) & (OZ_TNC - 1));
        const int eb = (col < P.N) ? P.eB[col] : 0;
        double v = fma((double)Phi[i], 268435456.0, (double)Plo[i]);
        v = (ea == OZ_BAD || eb == OZ_BAD) ? __longlong_as_double(0x7ff8000000000000ll) : ldexp(v, ea + eb - 63);
        stage[il * OZ_STAGE_LD + c0 + i] = v;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(32 * OZ_DW) : "memory");
      const int tid = threadIdx.x;
      for (int e = tid; e < OZ_TM * OZ_TNC; e += 32 * OZ_DW) {
        const int r = e / OZ_TNC, cc = e % OZ_TNC;
        const int i = mt * OZ_TM + r, jj = nt * OZ_TNC + cc;
        if (i >= P.M || jj >= P.N || (P.herm && jj > i)) continue;
        double f = P.alpha;
        if (P.s_row) f *= P.s_row[i / P.row_div];
        if (P.s_col) f *= P.s_col[jj / P.col_div];
        double2 val = make_double2(stage[r * OZ_STAGE_LD + cc] * f, stage[r * OZ_STAGE_LD + OZ_TNC + cc] * f);
        if (P.Creal) {  // real result (real operands): only the real part is stored
          double* dst = P.Creal + (long long)i * P.ldc + jj;
          if (P.beta) val.x += *dst;
          *dst = val.x;
        } else {
          double2* dst = P.C + (long long)i * P.ldc + jj;
          if (P.beta) {
            const double2 old = *dst;
            val.x += old.x;
            val.y += old.y;
          }
          *dst = val;
        }
        stage[r * OZ_STAGE_LD + cc] = val.x;  // the final value, for the mirror below
        stage[r * OZ_STAGE_LD + OZ_TNC + cc] = val.y;
      }
      if (P.herm) {  // mirror the strictly lower part: C[j][i] = conj(C[i][j])
        asm volatile("bar.sync 1, %0;" ::"r"(32 * OZ_DW) : "memory");
        for (int e = tid; e < OZ_TM * OZ_TNC; e += 32 * OZ_DW) {
          const int cc = e / OZ_TM, r = e % OZ_TM;
          const int i = mt * OZ_TM + r, jj = nt * OZ_TNC + cc;
          if (i >= P.M || jj >= P.N || jj >= i) continue;
          if (P.Creal) P.Creal[(long long)jj * P.ldc + i] = stage[r * OZ_STAGE_LD + cc];
          else
            P.C[(long long)jj * P.ldc + i] =
                make_double2(stage[r * OZ_STAGE_LD + cc], -stage[r * OZ_STAGE_LD + OZ_TNC + cc]);
        }
      }
    }
  }
  __syncthreads();
  if (*fail_sh && threadIdx.x == 0 && gb.status) atomicExch(gb.status, -6);  // TEBD_ERR_TIMEOUT
  if (warp == OZ_DW + 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
  }
}

struct Geo {
  int nkt, nrbA, nrbB;
  size_t plane_a, plane_b, offD1, offD2, offEA, offEB, total;
};

Geo geometry(int M, int N, int K, bool gram) {
  Geo g{};
  g.nkt = (K + 31) / 32;
  g.nrbA = 4 * ((M + OZ_TM - 1) / OZ_TM);
  g.nrbB = gram ? g.nrbA : (N + 31) / 32;
  g.plane_a = (size_t)OZ_S * g.nkt * g.nrbA * OZ_BLK;
  g.plane_b = (size_t)OZ_S * g.nkt * g.nrbB * OZ_BLK;
  g.offD1 = g.plane_a;
  g.offD2 = gram ? g.plane_a : g.offD1 + g.plane_b;
  g.offEA = g.offD2 + g.plane_b;
  g.offEB = g.offEA + (size_t)4 * 32 * g.nrbA;
  g.total = g.offEB + (gram ? 0 : (size_t)4 * 32 * g.nrbB) + 256;
  return g;
}

}  // namespace

static_assert(sizeof(OzGemmBatch) < 4000, "kernel parameter block too large");
static_assert(sizeof(OzPackBatch) < 4000, "kernel parameter block too large");
static_assert(bf16_idesc(128, 64) == ((1u << 4) | (1u << 7) | (1u << 10) | (8u << 17) | (8u << 24)), "idesc");

size_t oz_workspace_bytes(int M, int N, int K, bool gram) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  return geometry(M, N, K, gram).total;
}

int oz_gemm_launch(const std::vector<OzProb>& probs, int* status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    attr = true;
  }
  int launches = 0;
  size_t i0 = 0;
  while (i0 < probs.size()) {
    const size_t i1 = std::min(probs.size(), i0 + (size_t)OZ_MAXP);
    // row exponents and digits of every operand
    OzPackBatch eb{}, pk{};
    OzGemmBatch gb{};
    gb.status = status;
    int eblocks = 0, pblocks = 0, tiles = 0;
    auto add_job = [&](OzPackBatch& b, int& blocks, const OzPackJob& J, int per_job_blocks) {
      b.job[b.njob] = J;
      b.block_start[b.njob] = blocks;
      blocks += per_job_blocks;
      b.njob++;
    };
    for (size_t i = i0; i < i1; ++i) {
      const OzProb& p = probs[i];
      if (p.M <= 0 || p.N <= 0 || p.K <= 0) continue;
      const bool gram = p.gram != 0;
      const Geo g = geometry(p.M, p.N, p.K, gram);
      uint8_t* ws = reinterpret_cast<uint8_t*>(p.ws);
      uint16_t* DA = reinterpret_cast<uint16_t*>(ws);
      uint16_t* D1 = reinterpret_cast<uint16_t*>(ws + g.offD1);
      uint16_t* D2 = reinterpret_cast<uint16_t*>(ws + g.offD2);
      int* eA = reinterpret_cast<int*>(ws + g.offEA);
      int* eB = gram ? eA : reinterpret_cast<int*>(ws + g.offEB);
      OzPackJob ja{};
      ja.X = p.a.X; ja.rs = p.a.rs; ja.ks = p.a.ks; ja.scale = p.a.scale; ja.scale_div = std::max(1, p.a.scale_div);
      ja.conj = p.a.conj; ja.real = p.a.real; ja.rows = p.M; ja.K = p.K; ja.nrb = g.nrbA; ja.nkt = g.nkt; ja.e = eA;
      ja.P0 = DA; ja.type0 = 0;
      if (gram) {  // b = conj(a): D1 = digits of (ar, ai) = DA, D2 = (-ai, ar)
        ja.P1 = D2; ja.type1 = 3;
      }
      add_job(eb, eblocks, ja, g.nrbA);
      add_job(pk, pblocks, ja, g.nrbA * g.nkt);
      if (!gram) {
        OzPackJob jb{};
        jb.X = p.b.X; jb.rs = p.b.rs; jb.ks = p.b.ks; jb.scale = p.b.scale; jb.scale_div = std::max(1, p.b.scale_div);
        jb.conj = p.b.conj; jb.real = p.b.real; jb.rows = p.N; jb.K = p.K; jb.nrb = g.nrbB; jb.nkt = g.nkt; jb.e = eB;
        jb.P0 = D1; jb.type0 = 1;
        jb.P1 = D2; jb.type1 = 2;
        add_job(eb, eblocks, jb, g.nrbB);
        add_job(pk, pblocks, jb, g.nrbB * g.nkt);
      }
      OzTile& t = gb.p[gb.nprob];
      t.DA = DA; t.D1 = gram ? DA : D1; t.D2 = D2; t.eA = eA; t.eB = eB;
      t.C = p.C; t.Creal = p.Creal; t.ldc = p.ldc; t.alpha = p.alpha; t.s_row = p.s_row; t.s_col = p.s_col;
      t.row_div = std::max(1, p.row_div); t.col_div = std::max(1, p.col_div);
      t.M = p.M; t.N = p.N; t.nkt = g.nkt; t.nrbA = g.nrbA; t.nrbB = g.nrbB; t.herm = p.herm; t.beta = p.beta;
      t.tiles_n = (p.N + OZ_TNC - 1) / OZ_TNC;
      const int tm = (p.M + OZ_TM - 1) / OZ_TM;
      int nt_tiles = 0;
      if (p.herm) {
        for (int mt = 0; mt < tm; ++mt) nt_tiles += std::min(t.tiles_n, (mt * OZ_TM + OZ_TM - 1) / OZ_TNC + 1);
      } else {
        nt_tiles = tm * t.tiles_n;
      }
      gb.tile_start[gb.nprob] = tiles;
      tiles += nt_tiles;
      gb.nprob++;
    }
    eb.block_start[eb.njob] = eblocks;
    pk.block_start[pk.njob] = pblocks;
    gb.tile_start[gb.nprob] = tiles;
    if (tiles > 0) {
      k_oz_exp<<<eblocks, 256, 0, s>>>(eb);
      k_oz_pack<<<pblocks, 256, 0, s>>>(pk);
      k_oz_gemm<<<tiles, OZ_NT, OZ_SMEM, s>>>(gb);
      launches += 3;
    }
    i0 = i1;
  }
  return launches;
}

}  // namespace ptebd
