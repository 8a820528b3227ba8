// Recovery of the mixed form on the tensor cores (tcgen05):
//   u_T = P_T f_T - G_T^T lam_T   (eq. (12) after static condensation, Sec. 2.4)
// written as one product per triangle, u_T = [P_T, -G_T^T] [f_T; lam_T]: a GEMM over all
// triangles of a geometry class with the class operator as the shared operand
// (M = 128 triangles per tile, K = n_u + 3(k+1) padded to 16 or 32, N = n_u padded).
//
// Precision. bf16 products with FP32 accumulation carry 8 bits; the mixed form needs
// about 44. Each operand is therefore split into S = 7 signed 8-bit digits with one
// power-of-two scale per row (A: the triangle's f and lam) or per column (B: the class
// operator, split on the host): v = 2^e sum_s d_s 2^(-8(s+1)), |d_s| <= 256 (exact in
// bf16). The product of two digits is an integer below 2^16, so the sums over K = 32 and
// over the digit pairs (s, t) of one level L = s + t stay below 2^24 and the FP32
// accumulation in TMEM is exact. Levels L < S are accumulated (sum_L (L+1) = 28
// digit-pair products, 56 MMAs of K = 16), each in its own TMEM columns, and combined in
// double-float with the scales: the dropped levels L >= S bound the relative error by
// about (S+1) K 2^(-8S) = 4e-15 of max|row| max|column|.
//
// One CTA of 128 threads per tile: every thread slices its triangle's row into shared
// memory (canonical K-major core-matrix layout, no swizzle), one thread issues the MMAs
// and commits them to an mbarrier, and every warp reads its 32 TMEM lanes (its 32
// triangles) back. The mbarrier wait is bounded; TMEM is always released.
#include <cstdint>

#include <cuda_bf16.h>

#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"

namespace dgdf {

namespace {

constexpr int kTcThreads = 128;
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
  static constexpr int A_BYTES = kTcThreads * KP * 2;   // one digit slice of the A tile
  static constexpr int B_BYTES = NP * KP * 2;           // one digit slice of B
  static constexpr int SMEM = S * (A_BYTES + B_BYTES) + 256;
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

// Byte offset of element (row, k) in a K-major no-swizzle tile with KP columns: core matrix
// (row / 8, k / 8) holds 8 rows of 16 bytes; core matrices along K are 128 bytes apart, 8-row
// groups KP / 8 * 128 bytes apart.
template <int KP>
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return uint32_t((row >> 3) * (KP / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int K>
__global__ void __launch_bounds__(kTcThreads) k_recover_tc(DevMesh m, double* out, float2* out_df) {
  using T = TcShape<K>;
  constexpr int ND = T::ND, NL = Dims<K>::NL, KP = T::KP, NP = T::NP, S = T::S;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;                                 // S slices of [128][KP] bf16
  uint8_t* sB = smem + S * T::A_BYTES;                // S slices of [NP][KP] bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + S * T::B_BYTES);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 1);
  int* ok_s = reinterpret_cast<int*>(taddr_s + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = blockIdx.x;
  const int cls = __ldg(&m.tc_tile_cls[tile]);
  const int t = __ldg(&m.tc_rows[size_t(tile) * kTcThreads + tid]);   // -1: padding row

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
  // B: the class operator's digit slices, laid out on the host in this tile format
  {
    const uint4* src = reinterpret_cast<const uint4*>(m.tc_b) + size_t(cls) * (S * T::B_BYTES / 16);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < S * T::B_BYTES / 16; i += kTcThreads) dst[i] = __ldg(&src[i]);
  }
  // A: this thread's row [f_T; lam_T] as double-float, its scale and its digit slices
  int er = 0;
  {
    dfl a[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) a[k] = dfl(0);
    if (t >= 0) {
#pragma unroll
      for (int i = 0; i < ND; ++i) a[i] = to_dfl(m.h_df[size_t(t) * ND + i]);
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int f = __ldg(&m.tri_facet[size_t(t) * 3 + e]);
        const bool flip = __ldg(&m.tri_orient[size_t(t) * 3 + e]) < 0;
#pragma unroll
        for (int mm = 0; mm < NL; ++mm) {
          const dfl v = m.lam_is_df ? to_dfl(__ldcg(&m.lam_df[size_t(f) * m.lat_vs + mm]))
                                    : dfl(__ldcg(&m.lam[size_t(f) * NL + mm]));
          a[ND + e * NL + mm] = (flip && (mm & 1)) ? -v : v;
        }
      }
    }
    float amax = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) amax = fmaxf(amax, fabsf(a[k].hi));
    if (amax > 0.f) frexpf(amax, &er);
    // digits: t_0 = a 2^-er in [-1, 1]; d_s = rint(256 t_s), t_(s+1) = 256 t_s - d_s
#pragma unroll
    for (int k = 0; k < KP; ++k) a[k] = dfl(ldexpf(a[k].hi, -er), ldexpf(a[k].lo, -er));
#pragma unroll
    for (int s = 0; s < S; ++s) {
      uint32_t packed[KP / 2];
#pragma unroll
      for (int k = 0; k < KP; k += 2) {
        float d2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float x = a[k + q].hi * 256.f, y = a[k + q].lo * 256.f;
          const float d = rintf(x);
          float h, l;
          two_sum(x - d, y, h, l);   // exact: x - d is exact, the pair keeps the rest
          a[k + q] = dfl(h, l);
          d2[q] = d;
        }
        const __nv_bfloat16 b0 = __float2bfloat16_rn(d2[0]), b1 = __float2bfloat16_rn(d2[1]);
        packed[k / 2] = uint32_t(__bfloat16_as_ushort(b0)) | (uint32_t(__bfloat16_as_ushort(b1)) << 16);
      }
      uint8_t* base = sA + s * T::A_BYTES;
#pragma unroll
      for (int c = 0; c < KP / 8; ++c)
        *reinterpret_cast<uint4*>(base + core_off<KP>(tid, 8 * c)) =
            make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
    }
  }
  // operands visible to the tensor cores, TMEM address visible to every thread
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *taddr_s;
  if (tid == 0) {
    constexpr uint32_t idesc = idesc_bf16(kTcThreads, NP);
    constexpr uint32_t LBO = 128, SBO = (KP / 8) * 128;
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    for (int L = 0; L < S; ++L) {
      uint32_t acc = 0;
      for (int s = 0; s <= L; ++s) {
        const int tt = L - s;
#pragma unroll
        for (int kk = 0; kk < KP / 16; ++kk) {
          const uint64_t ad = smem_desc(a0 + s * T::A_BYTES + kk * 256, LBO, SBO);
          const uint64_t bd = smem_desc(b0 + tt * T::B_BYTES + kk * 256, LBO, SBO);
          tc_mma(tmem + uint32_t(L * NP), ad, bd, idesc, acc);
          acc = 1;
        }
      }
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
  if (ok) {
    // u[n] = sum_L 2^(er + ec[n] - 8 (L + 2)) D_L[n], smallest levels first
    dfl u[ND];
#pragma unroll
    for (int n = 0; n < ND; ++n) u[n] = dfl(0);
    const int* ec = m.tc_ec + cls * NP;
    const uint32_t lane_base = uint32_t(warp * 32) << 16;
    for (int L = S - 1; L >= 0; --L) {
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + lane_base + uint32_t(L * NP + c0), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          if (n < ND) u[n] = u[n] + dfl(ldexpf(__uint_as_float(r[j]), er + __ldg(&ec[n]) - 8 * (L + 2)), 0.f);
        }
      }
    }
    if (t >= 0) {
#pragma unroll
      for (int n = 0; n < ND; ++n) {
        if (out_df) out_df[size_t(t) * ND + n] = to_float2(u[n]);
        if (out) out[size_t(t) * ND + n] = to_double(u[n]);
      }
    }
  } else if (tid == 0) {
    atomicOr(&m.stats->flags, kFlagBarrierTimeout);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

template <int K>
cudaError_t launch_tc(const DevMesh& m, double* out, float2* out_df, cudaStream_t s) {
  using T = TcShape<K>;
  // at most two CTAs per SM, so that their TMEM (2 x 256 columns) always fits
  static bool attr = false;
  const int smem = 100 * 1024;
  static_assert(T::SMEM <= smem, "tile does not fit the requested shared memory");
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_recover_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_recover_tc<K><<<m.tc_tiles, kTcThreads, smem, s>>>(m, out, out_df);
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
