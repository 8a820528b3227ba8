// Recovery of the mixed form on the tensor cores (tcgen05):
//   u_T = P_T f_T - G_T^T lam_T   (eq. (12) after static condensation, Sec. 2.4)
// written as one product per triangle, u_T = [P_T, -G_T^T] [f_T; lam_T]: a GEMM over all
// triangles of a geometry class with the class operator as the shared operand
// (M = 128 triangles per tile, K = n_u + 3(k+1) padded to 16 or 32, N = n_u padded).
//
// The MMAs: one per A digit slice and K-chunk (14), N = S n_u columns: the B operand is a
// stack of S-1 zero blocks and the S digit slices of B, read from block S-1-s for A slice s,
// so that output column block j receives the digit pairs (s, j-s) of level j.
//
// Precision. bf16 products with FP32 accumulation carry 8 bits; the mixed form needs
// about 44. Each operand is therefore split into S = 7 signed 8-bit digits with one
// power-of-two scale per row (A: the triangle's f and lam) or per column (B: the class
// operator, split on the host): v = 2^e sum_s d_s 2^(-8(s+1)), |d_s| <= 256 (exact in
// bf16). The product of two digits is an integer below 2^16, so the sums over K = 32 and
// over the digit pairs (s, t) of one level L = s + t stay below 2^24 and the FP32
// accumulation in TMEM is exact. Levels L < S are accumulated (sum_L (L+1) = 28
// digit-pair products), each in its own TMEM columns, and combined in
// double-float with the scales: the dropped levels L >= S bound the relative error by
// about (S+1) K 2^(-8S) = 4e-15 of max|row| max|column|.
//
// One CTA of 512 threads per tile (two CTAs per SM: 32 warps hide the gathers' latency):
// four threads slice each triangle's row into shared memory (canonical K-major
// core-matrix layout, no swizzle), one thread issues the MMAs and commits them to an
// mbarrier, and warp w reads TMEM lanes 32 (w % 4) .. + 31 (its triangles) for column group
// w / 4 back. The mbarrier wait is bounded; TMEM is always released.
#include <cstdint>

#include <cuda_bf16.h>

#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"

namespace dgdf {

namespace {

constexpr int kTcRows = 128;          // triangles per tile (MMA M)
constexpr int kTcBlock = 512;         // threads per CTA: four per row while slicing
constexpr int kTcSlices = 7;          // digits per operand
constexpr uint32_t kTcTmemCols = 256;
constexpr unsigned long long kTcSpinLimit = 1ull << 20;

template <int K>
struct TcShape {
  static constexpr int ND = Dims<K>::ND, L3 = 3 * Dims<K>::NL;
  static constexpr int KR = ND + L3;                    // 12, 21, 32
  static constexpr int KP = KR <= 16 ? 16 : 32;         // padded K
  static constexpr int NP = ND <= 16 ? 16 : 32;         // padded N
  static constexpr int S = kTcSlices;
  static constexpr int A_BYTES = kTcRows * KP * 2;      // one digit slice of the A tile
  static constexpr int B_BYTES = NP * KP * 2;           // one digit slice of B
  static constexpr int RS = ND + 1;                     // padded row of the staging tile (float2)
  static_assert(kTcRows * RS * 8 <= S * A_BYTES, "the output tile reuses the A slices");
  // A slices (later the output tile) | S-1 zero blocks and the S digit slices of B | mbarrier, rows
  static constexpr int SMEM = S * A_BYTES + (2 * S - 1) * B_BYTES + 2048;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout of 8 x 16-byte core
// matrices; lbo = byte distance between core matrices adjacent along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;   // descriptor version (fixed 0b001 in bits 46-48)
  return d;                              // base offset 0, relative LBO, swizzle mode 0
}

// Instruction descriptor of kind::f16: A and B bf16, D f32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// 2^e as a float for -126 <= e <= 127 (built from its exponent field: exact)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
// v 2^e, exact while the result is a normal float (two factors keep each in range)
__device__ __forceinline__ float scale2(float v, int e) {
  const int e1 = e / 2;
  return v * pow2f(e1) * pow2f(e - e1);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with KP columns: core matrix
// (row / 8, k / 8) holds 8 rows of 16 bytes; core matrices along K are 128 bytes apart, 8-row
// groups KP / 8 * 128 bytes apart.
template <int KP>
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return uint32_t((row >> 3) * (KP / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int K>
__global__ void __launch_bounds__(kTcBlock, 2) k_recover_tc(DevMesh m, double* out, float2* out_df) {
  using T = TcShape<K>;
  constexpr int ND = T::ND, NL = Dims<K>::NL, L3 = T::L3, KP = T::KP, NP = T::NP, S = T::S, RS = T::RS;
  constexpr int KQ = KP / 4;        // A values sliced per thread (4 threads per row)
  constexpr int NG = NP / 8;        // column groups of 8 read back per level
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;                                      // S slices of [128][KP] bf16
  uint8_t* sB = smem + S * T::A_BYTES;                     // 2S-1 blocks of [NP][KP] bf16
  float2* sIO = reinterpret_cast<float2*>(sA);             // [128][RS] u, once the MMAs are done
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + (2 * S - 1) * T::B_BYTES);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 1);
  int* ok_s = reinterpret_cast<int*>(taddr_s + 1);
  int* rows_s = ok_s + 1;                                  // [128]
  int* er_s = rows_s + kTcRows;                            // [128] row exponents
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int cls = __ldg(&m.tc_tile_cls[tile]);
  if (tid < kTcRows) rows_s[tid] = __ldg(&m.tc_rows[size_t(tile) * kTcRows + tid]);   // -1: padding

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *ok_s = 1;
  }
  // B: S-1 zero blocks, then the class operator's S digit slices (laid out on the host). The
  // MMA of A slice s reads the N = S NP rows starting at block S-1-s, so that its column block
  // j meets B slice j - s (zero for j < s): column block j accumulates digit level j.
  __syncthreads();   // rows_s
  {
    const uint4* src = reinterpret_cast<const uint4*>(m.tc_b) + size_t(cls) * (S * T::B_BYTES / 16);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    constexpr int nz = (S - 1) * T::B_BYTES / 16, nb = S * T::B_BYTES / 16;
    for (int i = tid; i < nz; i += kTcBlock) dst[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < nb; i += kTcBlock) dst[nz + i] = __ldg(&src[i]);
  }
  __syncthreads();
  // A: row r = tid / 4, values k = KQ q .. KQ q + KQ - 1 (q = tid % 4) of [f_T; lam_T] (the four
  // lanes of a row read its f contiguously); the row scale is the maximum over the four lanes;
  // each digit slice is one 16-byte store
  {
    const int r = tid >> 2, q = tid & 3;
    const int tr = rows_s[r];
    // addresses first, then every load at once (no load behind a branch, so that they overlap):
    // f from the recovery input, the multipliers of the row's facets with the sign of the
    // facet's traversal for odd modes
    int fac[3];
    bool flp[3];
    const int trv = tr >= 0 ? tr : 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      fac[e] = __ldg(&m.tri_facet[size_t(trv) * 3 + e]);
      flp[e] = __ldg(&m.tri_orient[size_t(trv) * 3 + e]) < 0;
    }
    dfl a[KQ];
    bool neg[KQ], use[KQ];
    size_t idx[KQ];
    bool is_f[KQ];
#pragma unroll
    for (int j = 0; j < KQ; ++j) {
      const int k = KQ * q + j;
      // k < ND: f; ND <= k < ND + L3: multiplier mode mm of local facet fe; beyond: padding, which
      // reads a valid f entry of the row and is zeroed
      const bool lam_k = k >= ND && k < ND + L3;
      const int kl = lam_k ? k - ND : 0, fe = kl / NL, mm = kl - fe * NL;
      is_f[j] = !lam_k;
      use[j] = tr >= 0 && k < ND + L3;
      neg[j] = lam_k && (mm & 1) && flp[fe];
      const int f = fe == 0 ? fac[0] : (fe == 1 ? fac[1] : fac[2]);
      idx[j] = lam_k ? size_t(f) * (m.lam_is_df ? m.lat_vs : NL) + mm : size_t(trv) * ND + min(k, ND - 1);
    }
    if (m.lam_is_df) {
      float2 raw[KQ];
#pragma unroll
      for (int j = 0; j < KQ; ++j) raw[j] = __ldcg(is_f[j] ? &m.h_df[idx[j]] : &m.lam_df[idx[j]]);
#pragma unroll
      for (int j = 0; j < KQ; ++j) {
        const dfl v = to_dfl(raw[j]);
        a[j] = use[j] ? (neg[j] ? -v : v) : dfl(0);
      }
    } else {
      float2 rf[KQ];
      double rl[KQ];
#pragma unroll
      for (int j = 0; j < KQ; ++j) {
        rf[j] = __ldcg(&m.h_df[is_f[j] ? idx[j] : 0]);
        rl[j] = __ldcg(&m.lam[is_f[j] ? 0 : idx[j]]);
      }
#pragma unroll
      for (int j = 0; j < KQ; ++j) {
        const dfl v = is_f[j] ? to_dfl(rf[j]) : dfl(rl[j]);
        a[j] = use[j] ? (neg[j] ? -v : v) : dfl(0);
      }
    }
    float amax = 0.f;
#pragma unroll
    for (int j = 0; j < KQ; ++j) amax = fmaxf(amax, fabsf(a[j].hi));
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 2));
    // er: amax < 2^er <= 2 amax, from the exponent field (clamped: values near the top of the
    // float range have overflowed anyway)
    int er = amax > 0.f ? ((__float_as_int(amax) >> 23) & 0xff) - 126 : 0;
    er = min(er, 126);
    if (q == 0) er_s[r] = er;
    // digits: t_0 = a 2^-er in [-1, 1]; d_s = rint(256 t_s), t_(s+1) = 256 t_s - d_s
    const float sc = pow2f(-er);   // |er| <= 127 for any finite row maximum that is a normal float
#pragma unroll
    for (int j = 0; j < KQ; ++j) a[j] = dfl(a[j].hi * sc, a[j].lo * sc);
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      uint32_t packed[KQ / 2];
#pragma unroll
      for (int j = 0; j < KQ; j += 2) {
        float d2[2];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const float x = a[j + h2].hi * 256.f, y = a[j + h2].lo * 256.f;
          const float d = rintf(x);
          float hh, ll;
          two_sum(x - d, y, hh, ll);   // exact: x - d is exact, the pair keeps the rest
          a[j + h2] = dfl(hh, ll);
          d2[h2] = d;
        }
        const __nv_bfloat16 b0 = __float2bfloat16_rn(d2[0]), b1 = __float2bfloat16_rn(d2[1]);
        packed[j / 2] = uint32_t(__bfloat16_as_ushort(b0)) | (uint32_t(__bfloat16_as_ushort(b1)) << 16);
      }
      uint8_t* base = sA + sl * T::A_BYTES;
#pragma unroll
      for (int c = 0; c < KQ / 8; ++c)
        *reinterpret_cast<uint4*>(base + core_off<KP>(r, KQ * q + 8 * c)) =
            make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
      if constexpr (KQ == 4) {   // K = 16: half a core-matrix row per thread
        *reinterpret_cast<uint2*>(base + core_off<KP>(r, KQ * q)) = make_uint2(packed[0], packed[1]);
      }
    }
  }
  // operands visible to the tensor cores, TMEM address visible to every thread
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *taddr_s;
  if (tid == 0) {
    constexpr uint32_t idesc = idesc_bf16(kTcRows, S * NP);
    constexpr uint32_t LBO = 128, SBO = (KP / 8) * 128;
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    uint32_t acc = 0;
#pragma unroll 1
    for (int sl = 0; sl < S; ++sl)
#pragma unroll
      for (int kk = 0; kk < KP / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + sl * T::A_BYTES + kk * 256, LBO, SBO);
        const uint64_t bd = smem_desc(b0 + (S - 1 - sl) * T::B_BYTES + kk * 256, LBO, SBO);
        tc_mma(tmem, ad, bd, idesc, acc);
        acc = 1;
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
  }
  // wait for the MMAs (bounded: on time-out the tile writes nothing and the host sees the flag)
  {
    unsigned long long spins = 0;
    while (!mbar_try_wait(smem_u32(mbar), 0)) {
      if (++spins > kTcSpinLimit) {
        *ok_s = 0;
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const bool ok = *ok_s != 0;
  // read-back: warp w owns TMEM lanes 32 (w % 4) .. + 31 (rows) and column group w / 4 of
  // every level; u[n] = sum_L 2^(er + ec[n] - 8 (L + 2)) D_L[n], smallest levels first
  if (ok && warp / 4 < NG) {
    const int r = 32 * (warp & 3) + lane, g = warp >> 2;
    const int er = er_s[r];
    const int* ec = m.tc_ec + cls * NP + 8 * g;
    dfl u[8];
    int ecj[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      u[j] = dfl(0);
      ecj[j] = __ldg(&ec[j]);
    }
    const uint32_t lane_base = uint32_t(32 * (warp & 3)) << 16;
#pragma unroll 1
    for (int L = S - 1; L >= 0; --L) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(tmem + lane_base + uint32_t(L * NP + 8 * g))
                   : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) u[j] = u[j] + dfl(scale2(__uint_as_float(v[j]), er + ecj[j] - 8 * (L + 2)), 0.f);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (8 * g + j < ND) sIO[r * RS + 8 * g + j] = to_float2(u[j]);
  }
  if (!ok && tid == 0) atomicOr(&m.stats->flags, kFlagBarrierTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  if (ok) {
    // coalesced writes of the tile's rows
    for (int e = tid; e < kTcRows * ND; e += kTcBlock) {
      const int r = e / ND, c = e - r * ND;
      const int tr = rows_s[r];
      if (tr < 0) continue;
      const float2 v = sIO[r * RS + c];
      if (out_df) out_df[size_t(tr) * ND + c] = v;
      if (out) out[size_t(tr) * ND + c] = to_double(v);
    }
  }
}

template <int K>
cudaError_t launch_tc(const DevMesh& m, double* out, float2* out_df, cudaStream_t s) {
  using T = TcShape<K>;
  // at most two CTAs per SM, so that their TMEM (2 x 256 columns) always fits
  static bool attr = false;
  const int smem = 110 * 1024;
  static_assert(T::SMEM <= smem, "tile does not fit the requested shared memory");
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_recover_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_recover_tc<K><<<m.tc_tiles, kTcBlock, smem, s>>>(m, out, out_df);
  return cudaGetLastError();
}

}  // namespace

int tc_dims(int k, int* kp, int* np) {
  switch (k) {
    case 1: *kp = TcShape<1>::KP; *np = TcShape<1>::NP; return 0;
    case 2: *kp = TcShape<2>::KP; *np = TcShape<2>::NP; return 0;
    case 3: *kp = TcShape<3>::KP; *np = TcShape<3>::NP; return 0;
    default: return -1;
  }
}

cudaError_t launch_recover_tc(const DevMesh& m, double* out, float2* out_df, cudaStream_t s) {
  if (!m.tc_rows || m.tc_tiles < 1) return cudaErrorInvalidValue;
  switch (m.k) {
    case 1: return launch_tc<1>(m, out, out_df, s);
    case 2: return launch_tc<2>(m, out, out_df, s);
    case 3: return launch_tc<3>(m, out, out_df, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgdf
