// FP64 matrix products on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands from shared memory, FP32 accumulators in tensor memory) by
// exact integer slicing, the scheme of ozaki.cuh mapped onto sm_103a's
// asynchronous MMA.
//
// One 64 x 64 output tile per CTA of 256 threads, K in chunks of TC_KC = 32:
//  * staging (all threads): every row of the A chunk and every column of the
//    B chunk is scaled by its largest binary exponent and cut into OZ_S = 7
//    digits of 7 bits (ozaki.cuh, oz_digits), written as BF16 into shared
//    memory in the canonical no-swizzle K-major layout of the tensor cores:
//    core matrices of 8 rows x 8 elements (128 contiguous bytes), core
//    (g, kg) at byte (g * 4 + kg) * 128 (g: 8-row group, kg: 8-deep k group).
//    Digit s of A occupies row groups 8s..8s+7 (A digit 7 is all zeros), digit
//    t of B column groups 8t..8t+7.  Chunks are double-buffered: the digits of
//    chunk c + 1 are cut while the MMAs of chunk c run.
//  * MMAs (one elected thread): M = 128 rows [A_2j ; A_2j+1] (two digits
//    stacked), N = 64 columns B_t, K = 16, for j = 0..3, t = 0..6 with
//    2j + t <= 8: 22 MMAs per 16-deep step.  The accumulator of the top half
//    (rows 0..63) collects digit pairs of weight 2j + t, the bottom half
//    (rows 64..127) weight 2j + 1 + t.  Tensor-memory column block c (64
//    columns each) takes the MMAs of top weight c for c = 0..4 and of every
//    top weight >= 5 for c = 5; so block c holds, exactly, weight c (top) and
//    c + 1 (bottom) for c <= 3 -- at most three digit pairs of at most
//    129 * 127 over 32 of K, below 2^21 -- and the weights 5..9 in FP32.
//    Every digit pair with s + t <= 8 is multiplied once.
//  * flush (all threads, after the chunk's MMAs completed, signalled by
//    tcgen05.commit on an mbarrier): warp w reads tensor-memory lanes
//    32 (w % 4) .. 32 (w % 4) + 31 (the sub-partition it may access), i.e.
//    output rows from the top (w % 4 < 2) or bottom half, columns
//    32 (w / 4) .. + 31.  The exact weights are summed as a 64-bit integer in
//    units of 2^-28 times 2^8 and the FP32 part added in the same fixed
//    point; the top and bottom halves meet in shared memory, and each thread
//    keeps 16 outputs as (64-bit integer T, binary exponent S), T aligned to
//    the largest chunk scale so far by integer shifts.  FP64 arithmetic runs
//    once per output, at the end.
//
// Waits on the mbarrier are bounded; a wait that runs out sets *err (if
// given) to TC_TIMEOUT, waits once more (bounded) for the MMAs in flight,
// frees the tensor memory and leaves C unchanged.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "ozaki.cuh"

namespace aifmm {

constexpr int TC_KC = 32;                      // K chunk
constexpr int TC_KG = TC_KC / 8;               // 8-deep k groups per chunk
constexpr int TC_ABYTES = 64 * TC_KG * 128;    // A digits 0..7: 64 row groups
constexpr int TC_BBYTES = 56 * TC_KG * 128;    // B digits 0..6: 56 column groups
constexpr int TC_BUF = TC_ABYTES + TC_BBYTES;  // one chunk's operands
constexpr int TC_XBYTES = 256 * 16 * 8;        // top/bottom exchange
// dynamic shared memory: two operand buffers, the exchange, exponents, mbarrier
constexpr int TC_SMEM = 1024 + 2 * TC_BUF + TC_XBYTES + 2 * 2 * 64 * 4 + 64;
constexpr int TC_TIMEOUT = 9;
constexpr uint32_t TC_TMEM_COLS = 512;

__device__ inline uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// descriptor of a no-swizzle K-major operand starting at shared address a:
// leading (k) core-matrix stride 128 bytes, strided (row group) stride
// TC_KG * 128 bytes, descriptor version 1
__device__ inline uint64_t tc_desc(uint32_t a) {
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3ffff) >> 4);                  // start address, bits 0..13
  d |= (uint64_t)(128 >> 4) << 16;                      // leading byte offset, bits 16..29
  d |= (uint64_t)((TC_KG * 128) >> 4) << 32;            // stride byte offset, bits 32..45
  d |= (uint64_t)1 << 46;                               // version
  return d;                                             // base offset 0, no swizzle
}

// instruction descriptor: kind::f16, BF16 x BF16 -> F32, K-major A and B,
// M = 128, N = 64
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ inline void tc_mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc));
}

__device__ inline void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ inline bool tc_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity
__device__ inline bool tc_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (tc_try_wait(bar, parity)) return true;
  return false;
}

__device__ inline void tc_ld16(uint32_t ta, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}

// the integer of ozaki.cuh's split of x relative to the biased exponent
// E >= bexp(x): |x| = 2^(E - 1029) a 2^-42, a = round(m 2^(e - E - 4)) with
// the 53-bit mantissa m, a <= 2^49; the sign is returned separately
__device__ inline unsigned long long tc_int(double x, int E, bool& neg) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  neg = bits < 0;
  if (e == 0) return 0;
  const unsigned long long m = ((unsigned long long)bits & 0xfffffffffffffull) | (1ull << 52);
  const int sh = E - e + 4;
  return sh < 64 ? (m + (1ull << (sh - 1))) >> sh : 0;
}

// BF16 bit pattern of digit s of a (as ozaki.cuh's oz_digits: value d_s 2^(-7 s), signed)
__device__ inline uint32_t tc_digit(unsigned long long a, bool neg, int s) {
  const unsigned d = s == 0 ? (unsigned)(a >> 42) : (unsigned)((a >> (42 - 7 * s)) & 0x7f);
  const float v = __int_as_float((127 - 7 * s) << 23) * (float)d;     // d 2^(-7 s), exact
  return __bfloat16_as_ushort(__float2bfloat16_rn(neg ? -v : v));
}

// per output: running 64-bit fixed-point sum T at binary scale S (T 2^S in
// units of the digit products), aligned to the largest scale seen
__device__ inline void tc_accum(long long& T, int& S, long long t, int s) {
  if (t == 0) return;
  if (T == 0) {
    T = t;
    S = s;
    return;
  }
  if (s <= S) {
    const int d = S - s;
    if (d < 62) T += (t + (1ll << d >> 1)) >> d;
  } else {
    const int d = s - S;
    T = d < 62 ? (T + (1ll << d >> 1)) >> d : 0;
    S = s;
    T += t;
  }
}

// C[0..mr, 0..nc] += alpha * op(A)[0..mr, 0..K) B[0..K, 0..nc]; op(A) = A
// column-major (lda) or, with TA, A^T for A column-major K x mr (lda);
// B column-major (ldb), C column-major (ldc).  256 threads; smem: TC_SMEM
// bytes of dynamic shared memory (any alignment; aligned to 1024 here).
template <bool TA = false>
__device__ void tile_gemm_64_tc(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int mr,
                                int nc, int K, double alpha, unsigned char* smem_raw, int* err) {
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* buf0 = smem;                                            // [2][TC_BUF]
  long long* xch = reinterpret_cast<long long*>(smem + 2 * TC_BUF);      // [256][16]
  int* ex = reinterpret_cast<int*>(smem + 2 * TC_BUF + TC_XBYTES);      // [2][2][64]: ea, eb per buffer
  uint64_t* bar = reinterpret_cast<uint64_t*>(ex + 2 * 2 * 64);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (K <= 0) return;
  const int nchunk = (K + TC_KC - 1) / TC_KC;

  // ---- set-up: zero A digit 7 of both buffers, mbarrier, tensor memory
  for (int b = 0; b < 2; ++b)
    for (int e = tid; e < 8 * TC_KG * 128 / 16; e += 256)
      reinterpret_cast<uint4*>(buf0 + b * TC_BUF + 56 * TC_KG * 128)[e] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }

  // staging of chunk c into buffer c & 1: thread (x = tid % 64, g = tid / 64)
  // takes row x of op(A) and column x of B at k = 8g..8g+7 of the chunk
  const int sx = tid & 63, sg = tid >> 6;
  auto stage = [&](int c) {
    unsigned char* bf = buf0 + (c & 1) * TC_BUF;
    int* ea = ex + (c & 1) * 128;
    int* eb = ea + 64;
    const int k0 = c * TC_KC + 8 * sg;
    double av[8], bv[8];
    int am = 0, bm = 0;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = k0 + kk;
      double a = 0.0, b = 0.0;
      if (k < K) {
        if (sx < mr) a = TA ? A[k + (size_t)sx * lda] : A[sx + (size_t)k * lda];
        if (sx < nc) b = B[k + (size_t)sx * ldb];
      }
      av[kk] = a;
      bv[kk] = b;
      am = max(am, oz_bexp(a));
      bm = max(bm, oz_bexp(b));
    }
    // the previous use of this buffer's exponents ended with the flush of
    // chunk c - 2, before the barrier that closed it
    if (sg == 0) {
      ea[sx] = 0;
      eb[sx] = 0;
    }
    __syncthreads();
    atomicMax(&ea[sx], am);
    atomicMax(&eb[sx], bm);
    __syncthreads();
    const int Ea = ea[sx], Eb = eb[sx];
    unsigned long long ia[8], ib[8];
    unsigned na = 0, nb = 0;                               // sign bits
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      bool n1, n2;
      ia[kk] = tc_int(av[kk], Ea, n1);
      ib[kk] = tc_int(bv[kk], Eb, n2);
      na |= (unsigned)n1 << kk;
      nb |= (unsigned)n2 << kk;
    }
    // one 16-byte core-matrix row per digit: (group, kg = sg, row x % 8)
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      uint32_t qa[4], qb[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        qa[h] = tc_digit(ia[2 * h], (na >> (2 * h)) & 1, s) | (tc_digit(ia[2 * h + 1], (na >> (2 * h + 1)) & 1, s) << 16);
        qb[h] = tc_digit(ib[2 * h], (nb >> (2 * h)) & 1, s) | (tc_digit(ib[2 * h + 1], (nb >> (2 * h + 1)) & 1, s) << 16);
      }
      const int gi = s * 8 + (sx >> 3);
      *reinterpret_cast<uint4*>(bf + (gi * TC_KG + sg) * 128 + (sx & 7) * 16) = make_uint4(qa[0], qa[1], qa[2], qa[3]);
      *reinterpret_cast<uint4*>(bf + TC_ABYTES + (gi * TC_KG + sg) * 128 + (sx & 7) * 16) =
          make_uint4(qb[0], qb[1], qb[2], qb[3]);
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };

  stage(0);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const uint32_t barad = tc_smem_u32(bar);

  // outputs of this thread: row r (TMEM lane quarter q), 16 columns
  const int q = w & 3, hf = w >> 2;
  const bool top = q < 2;
  const int r = 32 * (q & 1) + lane;                       // output row
  // top threads finish columns 32 hf + 0..15, bottom threads 32 hf + 16..31
  const int cfin = 32 * hf + (top ? 0 : 16);
  long long T[16];
  int S[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    T[j] = 0;
    S[j] = 0;
  }
  bool ok = true;

  // 16 columns of this warp's lanes from every block, as fixed point in
  // units of 2^-36 of the digit products: exact weights << 8 plus the FP32 part
  auto gather16 = [&](uint32_t ta, long long (&pt)[16]) {
    long long tx[16];
    float fx[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      tx[j] = 0;
      fx[j] = 0.f;
    }
#pragma unroll
    for (int blk = 0; blk < 6; ++blk) {
      uint32_t v[16];
      tc_ld16(ta + 64 * blk, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int wgt = top ? blk : blk + 1;                  // weight of this half of the block
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float f = __uint_as_float(v[j]);
        if (blk < 5 && wgt <= 4)
          tx[j] += (long long)__float2int_rn(f * (float)(1 << (7 * wgt))) * (1ll << (7 * (4 - wgt)));
        else
          fx[j] += f;
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) pt[j] = tx[j] * 256 + __float2ll_rn(fx[j] * 68719476736.0f);
  };

  for (int c = 0; c < nchunk; ++c) {
    unsigned char* bf = buf0 + (c & 1) * TC_BUF;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t abase = tc_smem_u32(bf), bbase = abase + TC_ABYTES;
      bool first[6] = {true, true, true, true, true, true};
#pragma unroll
      for (int ks = 0; ks < TC_KC / 16; ++ks)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int t = 0; t < OZ_S; ++t) {
            if (2 * j + t > OZ_S + 1) continue;
            const int blk = min(2 * j + t, 5);
            const uint64_t ad = tc_desc(abase + ((16 * j) * TC_KG + 2 * ks) * 128);
            const uint64_t bd = tc_desc(bbase + ((8 * t) * TC_KG + 2 * ks) * 128);
            tc_mma(tbase + 64 * blk, ad, bd, first[blk] ? 0u : 1u);
            first[blk] = false;
          }
      tc_commit(barad);
    }
    if (c + 1 < nchunk) stage(c + 1);
    ok = __syncthreads_and(tc_wait(barad, c & 1) ? 1 : 0) != 0;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- flush: the half of the columns handed to the partner first
    const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + 32 * hf;
    {
      long long pt[16];
      gather16(ta + (top ? 16 : 0), pt);
#pragma unroll
      for (int j = 0; j < 16; ++j) xch[(size_t)tid * 16 + j] = pt[j];
    }
    long long pk[16];
    gather16(ta + (top ? 0 : 16), pk);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // partner: same row, other half of the accumulator, same column half
    const int ptid = tid ^ 64;                              // q <-> q ^ 2
    const int* ea = ex + (c & 1) * 128;
    const int* eb = ea + 64;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long tsum = pk[j] + xch[(size_t)ptid * 16 + j];
      // scale of the chunk: 2^(E_r - 1029) 2^(E_c - 1029) 2^-36 per unit
      tc_accum(T[j], S[j], tsum, ea[r] + eb[cfin + j]);
    }
    __syncthreads();   // exchange and exponents read before they are rewritten
  }

  if (!ok) {
    if (tid == 0 && err) atomicCAS(err, 0, TC_TIMEOUT);
    // the MMAs in flight: one more bounded wait on every phase not yet seen
    for (int c = 0; c < 2; ++c) tc_wait(barad, c & 1);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = cfin + j;
      if (r < mr && col < nc && T[j] != 0) {
        // T 2^(S - 2058 - 36): biased exponent of the scale S - 2058 - 36 + 1023
        const int be = S[j] - 2058 - 36 + 1023;
        double sc = 0.0;
        if (be > 0 && be < 2047) sc = __longlong_as_double((long long)be << 52);
        else if (be <= 0 && be > -52) sc = __longlong_as_double(1ll << (51 + be));   // subnormal
        C[r + (size_t)col * ldc] += alpha * ((double)T[j] * sc);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_TMEM_COLS));
  }
}

}  // namespace aifmm
