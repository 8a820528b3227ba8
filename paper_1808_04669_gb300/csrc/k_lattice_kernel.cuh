// Facet-system solve on translation-invariant split-square meshes (the lattice
// path of the condensed hybrid-mixed system, eq. (12) of Sec. 2.4).
//
// On such a mesh the facet operator S is block circulant over the N x N cell
// grid: a 2-D discrete Fourier transform turns it into one Hermitian block
// S^(kappa) of size C = 3(k+1) per wavenumber, and S^+ r = IDFT(S^(kappa)^+ DFT(r))
// (pseudo-inverse at kappa = 0, the constant multiplier). This kernel runs PCG
// preconditioned by that Fourier-space inverse:
//   FP64 form : FP64 vectors, FP64 SpMV, FP64 transforms (one or two iterations);
//   mixed form: double-float vectors and SpMV on the FP32 units, FP32 transforms
//               (a few iterations: the preconditioned operator is I + O(FP32 rounding)).
// The residual is real, so only the wavenumbers ki in [0, N/2] are transformed:
//   rows   : two facet rows j, j+1 packed as one complex row, FFT along i, split
//            into the two half spectra (Hermitian symmetry)
//   columns: per ki, FFT along j, multiply by S^(kappa)^+ (FP32: its near-singular
//            eigen-direction applied on its own plus the packed Hermitian remainder, so
//            FP32 rounding causes no cancellation), inverse FFT along j
//   rows   : inverse FFT along i of two rows packed the same way (scaled 1/N^2)
// with a grid barrier between the passes. Transforms run in shared memory: for N a
// power of two up to 1024 (FP32) / 256 (FP64) a two-pass FFT whose radix-sqrt(N)
// DFTs run in registers, self-sorting (Stockham) radix-2 passes for larger powers of
// two, a direct DFT otherwise. One persistent cooperative kernel per solve, two blocks
// per SM.
#pragma once

#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"
#include "solver_common.cuh"

namespace dgdf {
namespace {

constexpr int kLatThreads = 256;
constexpr int kLatTJ = 4;          // facet rows j per row-pass tile (two packed pairs)

template <bool MIXED>
struct LatT;
template <>
struct LatT<false> {   // FP64 form
  using R = double;
  using C2 = double2;
  using V = double;     // vector storage (lam, g, r, p, q)
  using A = double;     // arithmetic on vector values
  using Z = double;     // preconditioned residual z
  using Acc = double;
};
template <>
struct LatT<true> {    // mixed form
  using R = float;
  using C2 = float2;
  using V = float2;
  using A = dfl;
  using Z = float;
  using Acc = dacc;
};

// ---- typed vector access and accumulation
__device__ __forceinline__ double ldv(const double* p) { return __ldcg(p); }
__device__ __forceinline__ dfl ldv(const float2* p) { return to_dfl(__ldcg(p)); }
__device__ __forceinline__ double ldz(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldz(const float* p) { return __ldcg(p); }
__device__ __forceinline__ void stv(double* p, double v) { *p = v; }
__device__ __forceinline__ void stv(float2* p, dfl v) { *p = to_float2(v); }
__device__ __forceinline__ void mad(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void acc_add(double& a, double v) { a += v; }
__device__ __forceinline__ void acc_add(dacc& a, dfl v) {
  float s, t;
  two_sum(a.s, v.hi, s, t);
  a.s = s;
  a.c += t + v.lo;
}
__device__ __forceinline__ double acc_zero(double) { return 0.0; }
__device__ __forceinline__ dacc acc_zero(dacc) { return dacc_zero(); }
__device__ __forceinline__ double acc_val(double a) { return a; }
__device__ __forceinline__ double acc_val(const dacc& a) { return double(a.s) + double(a.c); }
__device__ __forceinline__ double fin(double a) { return a; }
__device__ __forceinline__ dfl fin(const dacc& a) { return val(a); }
__device__ __forceinline__ double fft_in(double v) { return v; }
__device__ __forceinline__ float fft_in(dfl v) { return v.hi; }
__device__ __forceinline__ double as_a(double v) { return v; }
__device__ __forceinline__ double lead_d(double v) { return v; }
__device__ __forceinline__ double lead_d(dfl v) { return double(v.hi); }
__device__ __forceinline__ dfl as_a(float v) { return dfl(v, 0.f); }
__device__ __forceinline__ double stencil_entry(const DevMesh& m, size_t i, double) { return __ldg(&m.st_blk[i]); }
__device__ __forceinline__ dfl stencil_entry(const DevMesh& m, size_t i, dfl) { return to_dfl(__ldg(&m.st_blk_df[i])); }

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C2>
__device__ __forceinline__ C2 cadd(C2 a, C2 b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename C2>
__device__ __forceinline__ C2 csub(C2 a, C2 b) {
  return {a.x - b.x, a.y - b.y};
}
// a += h b
template <typename C2>
__device__ __forceinline__ void cmad(C2& a, C2 h, C2 b) {
  a.x += h.x * b.x - h.y * b.y;
  a.y += h.x * b.y + h.y * b.x;
}
// a += conj(h) b
template <typename C2>
__device__ __forceinline__ void cmad_conj(C2& a, C2 h, C2 b) {
  a.x += h.x * b.x + h.y * b.y;
  a.y += h.x * b.y - h.y * b.x;
}

// Self-sorting (Stockham) radix-2 FFT of `rows` rows of length n = 2^logn, natural
// order in and out, ping-ponging between a and b; returns the buffer holding the
// result. Stage s combines pairs (j, j + n/2) of the input into outputs
// (j / l) 2l + j % l and that + l, l = 2^s, with twiddle exp(-+2 pi i (j % l) / (2l)).
// tw[t] = exp(-2 pi i t / n).
template <typename C2>
__device__ C2* fft_stockham(C2* a, C2* b, int rows, int logn, const C2* tw, bool inverse) {
  const int n = 1 << logn, hn = n >> 1;
  for (int s = 0; s < logn; ++s) {
    const int l = 1 << s;
#pragma unroll 4
    for (int e = threadIdx.x; e < rows * hn; e += blockDim.x) {
      const int row = e >> (logn - 1), j = e & (hn - 1);
      const C2* x = a + row * n;
      C2* y = b + row * n;
      const int k = j & (l - 1);
      C2 w = tw[k << (logn - 1 - s)];
      if (inverse) w.y = -w.y;
      const C2 c0 = x[j], c1 = cmul(x[j + hn], w);
      const int d = ((j - k) << 1) + k;
      y[d] = cadd(c0, c1);
      y[d + l] = csub(c0, c1);
    }
    __syncthreads();
    C2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// In-register DFT of size R (a power of two), natural order in and out: radix-2
// decimation in frequency with twiddles w^j = tw[j tstep] (w = exp(-+2 pi i / R)),
// then the bit-reversal permutation of the registers (resolved at compile time).
template <int R, typename C2>
__device__ __forceinline__ void reg_dft(C2 (&v)[R], const C2* tw, int tstep, bool inverse) {
#pragma unroll
  for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const C2 a = v[blk + j], b = v[blk + j + half];
        v[blk + j] = cadd(a, b);
        const C2 d = csub(a, b);
        if (j == 0) {
          v[blk + j + half] = d;
        } else {
          C2 w = tw[j * (R / (2 * half)) * tstep];
          if (inverse) w.y = -w.y;
          v[blk + j + half] = cmul(d, w);
        }
      }
    }
  }
  C2 t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int b = 0;
#pragma unroll
    for (int q = 1; q < R; q <<= 1) b = (b << 1) | ((i / q) & 1);
    t[i] = v[b];
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}

// Two-pass ("four-step") FFT of `rows` rows of length N = R1 R2 held in a (natural
// order, in place), through the scratch s (rows of stride R2 (R1 + 1), padded against
// bank conflicts): x[n1 + R1 n2] -> DFT over n2 (thread per (row, n1)) -> twiddle
// w_N^(n1 k2) -> DFT over n1 (thread per (row, k2)) -> X[k2 + R2 k1].
template <int R1, int R2, typename C2>
__device__ void fft_four_step(C2* a, C2* s, int rows, const C2* tw, bool inverse) {
  constexpr int N = R1 * R2, SR = R2 * (R1 + 1);
  for (int t = threadIdx.x; t < rows * R1; t += blockDim.x) {
    const int row = t / R1, n1 = t - row * R1;
    C2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = a[row * N + n1 + R1 * n2];
    reg_dft<R2>(v, tw, R1, inverse);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      C2 w = tw[n1 * k2];
      if (inverse) w.y = -w.y;
      s[row * SR + k2 * (R1 + 1) + n1] = k2 == 0 ? v[k2] : cmul(v[k2], w);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < rows * R2; t += blockDim.x) {
    const int row = t / R2, k2 = t - row * R2;
    C2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = s[row * SR + k2 * (R1 + 1) + n1];
    reg_dft<R1>(v, tw, R2, inverse);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[row * N + k2 + R2 * k1] = v[k1];
  }
  __syncthreads();
}

// Largest log2 N handled by the two-pass FFT (register budget of one radix-R pass).
template <typename C2>
struct FourStepMax;
template <>
struct FourStepMax<float2> {
  static constexpr int logn = 10;
};
template <>
struct FourStepMax<double2> {
  static constexpr int logn = 8;
};

// Direct DFT of `rows` rows of length n (any n): out[r][k] = sum_t in[r][t] w^(t k mod n),
// w[m] = exp(-2 pi i m / n) (conjugated for the inverse). Natural order in and out.
template <typename C2>
__device__ void dft(const C2* in, C2* out, int rows, int n, const C2* tw, bool inverse) {
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int row = e / n, k = e - row * n;
    const C2* x = in + row * n;
    C2 acc = {0, 0};
    int idx = 0;
    for (int t = 0; t < n; ++t) {
      C2 w = tw[idx];
      if (inverse) w.y = -w.y;
      acc = cadd(acc, cmul(x[t], w));
      idx += k;
      if (idx >= n) idx -= n;
    }
    out[e] = acc;
  }
  __syncthreads();
}

template <int K, bool MIXED>
struct LatCtx {
  using T = LatT<MIXED>;
  using C2 = typename T::C2;
  static constexpr int NL = K + 1, C = 3 * NL;
  // facet stride of the solver vectors: padded to 4 for k = 2 in the mixed form, so that
  // every facet's values are one aligned 16- or 32-byte access
  static constexpr int VS = (MIXED && NL == 3) ? 4 : NL;
  // stored entries per wavenumber: FP32, the deflated eigen form (the eigenvector v1 of the
  // largest inverse eigenvalue, that eigenvalue, the packed upper triangle of the rest);
  // FP64, the full inverse block
  static constexpr int NP = MIXED ? C + 1 + C * (C + 1) / 2 : C * C;
  int N, logn, NK, ntj;   // NK = N/2 + 1 wavenumbers ki; ntj row tiles per facet type
  int grp;                // rows transformed at a time (the scratch holds grp rows)
  bool pow2;              // FFT (N a power of two) or direct DFT
  C2* tw;                 // [N] exp(-2 pi i t / N)
  C2* bufa;               // transform data, max(C, 2(k+1)) rows of N
  C2* scr;                // scratch, grp rows of lattice_scratch_row(N)
  C2* X;                  // [C][NK][N] spectrum: half along i, full along j (then along kj)
  // split column pass (lattice_split): each column ki is two work items, the even and the
  // odd wavenumbers kj (one decimation-in-frequency step, then transforms of length N/2);
  // their inverse halves go to X2 and the inverse row pass adds them
  bool split;
  C2* tw2;                // [N/2] exp(-2 pi i t / (N/2))
  C2* X2;                 // [C][NK][N]: [0, N/2) the even half E, [N/2, N) w^-j times the odd half
  const C2* S;            // [NK][NP][N] S^(kappa)^+ (packed upper triangle or full), kj fastest
  // vectors, facet-major [n_facet][NL] in lattice order
  typename T::V *lam, *g, *r, *q;
  typename T::Z* z;
};

// Forward or inverse transform, in place, of `rows` natural-order rows held in a: groups
// of L.grp rows go through the scratch buffer. Powers of two up to FourStepMax: the
// two-pass FFT; larger powers of two: Stockham passes; other N: the direct DFT (both
// out of place; a result left in the scratch is copied back).
template <int K, bool MIXED>
__device__ void xform(const LatCtx<K, MIXED>& L, typename LatT<MIXED>::C2* a, int rows, bool inverse) {
  using C2 = typename LatT<MIXED>::C2;
  const int N = L.N;
  for (int r0 = 0; r0 < rows; r0 += L.grp) {
    const int gr = min(L.grp, rows - r0);
    C2* d = a + size_t(r0) * N;
    if (L.pow2 && L.logn <= FourStepMax<C2>::logn) {
      switch (L.logn) {
        case 0: break;
        case 1: fft_four_step<2, 1>(d, L.scr, gr, L.tw, inverse); break;
        case 2: fft_four_step<2, 2>(d, L.scr, gr, L.tw, inverse); break;
        case 3: fft_four_step<4, 2>(d, L.scr, gr, L.tw, inverse); break;
        case 4: fft_four_step<4, 4>(d, L.scr, gr, L.tw, inverse); break;
        case 5: fft_four_step<8, 4>(d, L.scr, gr, L.tw, inverse); break;
        case 6: fft_four_step<8, 8>(d, L.scr, gr, L.tw, inverse); break;
        case 7: fft_four_step<16, 8>(d, L.scr, gr, L.tw, inverse); break;
        case 8: fft_four_step<16, 16>(d, L.scr, gr, L.tw, inverse); break;
        default:
          if constexpr (FourStepMax<C2>::logn >= 10) {
            if (L.logn == 9) fft_four_step<32, 16>(d, L.scr, gr, L.tw, inverse);
            else fft_four_step<32, 32>(d, L.scr, gr, L.tw, inverse);
          }
          break;
      }
      continue;
    }
    const C2* res;
    if (L.pow2) {
      res = fft_stockham(d, L.scr, gr, L.logn, L.tw, inverse);
    } else {
      dft(d, L.scr, gr, N, L.tw, inverse);
      res = L.scr;
    }
    if (res != d) {
      for (int e = threadIdx.x; e < gr * N; e += blockDim.x) d[e] = res[e];
      __syncthreads();
    }
  }
}

// ---- one facet's NL values of a solver vector (facet stride VS), as aligned vector
// accesses where the stride allows (coherent L2 loads: the data was written by other
// blocks before the last grid barrier)
template <int NL, int VS>
__device__ __forceinline__ void ldf(const float2* p, dfl (&v)[NL]) {
  if constexpr (VS % 2 == 0) {
#pragma unroll
    for (int h = 0; h < VS / 2; ++h) {
      const float4 w = __ldcg(reinterpret_cast<const float4*>(p) + h);
      if (2 * h < NL) v[2 * h] = dfl(w.x, w.y);
      if (2 * h + 1 < NL) v[2 * h + 1] = dfl(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NL; ++j) v[j] = to_dfl(__ldcg(p + j));
  }
}
template <int NL, int VS>
__device__ __forceinline__ void stf(float2* p, const dfl (&v)[NL]) {
  if constexpr (VS % 2 == 0) {
#pragma unroll
    for (int h = 0; h < VS / 2; ++h) {
      const dfl a = (2 * h < NL) ? v[2 * h] : dfl(0), b = (2 * h + 1 < NL) ? v[2 * h + 1] : dfl(0);
      reinterpret_cast<float4*>(p)[h] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NL; ++j) p[j] = to_float2(v[j]);
  }
}
template <int NL, int VS>
__device__ __forceinline__ void ldf(const float* p, float (&v)[NL]) {
  if constexpr (VS == 4) {
    const float4 w = __ldcg(reinterpret_cast<const float4*>(p));
    const float t[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < NL; ++j) v[j] = t[j];
  } else if constexpr (VS == 2) {
    const float2 w = __ldcg(reinterpret_cast<const float2*>(p));
    v[0] = w.x;
    v[NL - 1] = w.y;
  } else {
#pragma unroll
    for (int j = 0; j < NL; ++j) v[j] = __ldcg(p + j);
  }
}
template <int NL, int VS>
__device__ __forceinline__ void stf(float* p, const float (&v)[NL]) {
  if constexpr (VS == 4) {
    float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NL; ++j) t[j] = v[j];
    *reinterpret_cast<float4*>(p) = make_float4(t[0], t[1], t[2], t[3]);
  } else if constexpr (VS == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[NL - 1]);
  } else {
#pragma unroll
    for (int j = 0; j < NL; ++j) p[j] = v[j];
  }
}
template <int NL, int VS>
__device__ __forceinline__ void ldf(const double* p, double (&v)[NL]) {
  if constexpr (VS % 2 == 0) {
#pragma unroll
    for (int h = 0; h < VS / 2; ++h) {
      const double2 w = __ldcg(reinterpret_cast<const double2*>(p) + h);
      if (2 * h < NL) v[2 * h] = w.x;
      if (2 * h + 1 < NL) v[2 * h + 1] = w.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < NL; ++j) v[j] = __ldcg(p + j);
  }
}
template <int NL, int VS>
__device__ __forceinline__ void stf(double* p, const double (&v)[NL]) {
  if constexpr (VS % 2 == 0) {
#pragma unroll
    for (int h = 0; h < VS / 2; ++h) reinterpret_cast<double2*>(p)[h] = make_double2(v[2 * h], v[2 * h + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < NL; ++j) p[j] = v[j];
  }
}

// Facets are numbered (type, j, i) on a lattice mesh, so a tile of kLatTJ rows of one
// facet type with all k+1 modes is one contiguous range of the facet-major vectors:
// DOF index ((type N + j) N + i) VS + m.

// Row pass, forward: per tile read r and update it: with `update`, r -= alpha q + c_prev 1 and
// lam += alpha_lam p (1 is the constant multiplier, mode 0 on every facet); without (the first
// pass of a solve, r holding g - S lam0), r = scale (r - c_prev 1), and the multiplier history
// moves down one slot (hdst <- hsrc, when hsrc is set). Accumulate r.r and the sum of the
// mode-0 entries of r, pack rows j0+2p (real part) and j0+2p+1 (imaginary part) per mode, FFT
// along i, split into the two rows' half spectra and store them in X.
template <int K, bool MIXED>
__device__ void rows_forward(const LatCtx<K, MIXED>& L, bool update, typename LatT<MIXED>::A alpha,
                             typename LatT<MIXED>::A alpha_lam, typename LatT<MIXED>::A c_prev,
                             const typename LatT<MIXED>::V* p, typename LatT<MIXED>::Acc& rr,
                             typename LatT<MIXED>::Acc& r0sum, typename LatT<MIXED>::A scale,
                             const typename LatT<MIXED>::V* hsrc, typename LatT<MIXED>::V* hdst) {
  using T = LatT<MIXED>;
  using C2 = typename T::C2;
  using R = typename T::R;
  using A = typename T::A;
  constexpr int NL = K + 1, VS = LatCtx<K, MIXED>::VS;
  const int N = L.N, NK = L.NK;
  const int ntiles = 3 * L.ntj;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ty = tile / L.ntj, j0 = (tile - ty * L.ntj) * kLatTJ;
    const int rows = min(kLatTJ, N - j0), npair = (rows + 1) >> 1;
    const size_t base = (size_t(ty) * N + j0) * N * VS;
#pragma unroll 4
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {   // one facet (row r_, column i)
      const int r_ = e / N, i = e - r_ * N;
      const size_t o = base + size_t(e) * VS;
      A rv[NL];
      ldf<NL, VS>(L.r + o, rv);
      if (update) {
        A qv[NL], lv[NL], pv[NL];
        ldf<NL, VS>(L.q + o, qv);
        ldf<NL, VS>(L.lam + o, lv);
        ldf<NL, VS>(p + o, pv);
#pragma unroll
        for (int mm = 0; mm < NL; ++mm) {
          rv[mm] = rv[mm] - alpha * qv[mm];
          lv[mm] = lv[mm] + alpha_lam * pv[mm];
        }
        rv[0] = rv[0] - c_prev;   // the constant-multiplier component measured last pass
        stf<NL, VS>(L.r + o, rv);
        stf<NL, VS>(L.lam + o, lv);
      } else {
        rv[0] = rv[0] - c_prev;
#pragma unroll
        for (int mm = 0; mm < NL; ++mm) rv[mm] = scale * rv[mm];
        stf<NL, VS>(L.r + o, rv);
        if (hsrc) {
          A hv[NL];
          ldf<NL, VS>(hsrc + o, hv);
          stf<NL, VS>(hdst + o, hv);
        }
      }
      acc_add(r0sum, rv[0]);
#pragma unroll
      for (int mm = 0; mm < NL; ++mm) {
        mad(rr, rv[mm], rv[mm]);
        C2* slot = &L.bufa[((r_ >> 1) * NL + mm) * N + i];
        if (r_ & 1) slot->y = fft_in(rv[mm]);
        else slot->x = fft_in(rv[mm]);
      }
    }
    if (rows & 1)   // the last pair has no odd row
      for (int e = threadIdx.x; e < NL * N; e += blockDim.x) L.bufa[((npair - 1) * NL) * N + e].y = R(0);
    __syncthreads();
    xform(L, L.bufa, npair * NL, false);
    const C2* res = L.bufa;
    // Z = X_even + i X_odd: X_even[k] = (Z[k] + conj Z[-k]) / 2, X_odd[k] = (Z[k] - conj Z[-k]) / (2i)
    for (int e = threadIdx.x; e < rows * NK * NL; e += blockDim.x) {
      const int r_ = e % rows, rest = e / rows;
      const int ki = rest % NK, mm = rest / NK;
      const C2* row = res + ((r_ >> 1) * NL + mm) * N;
      const C2 Z = row[ki], Zc = row[ki == 0 ? 0 : N - ki];
      C2 out;
      if (r_ & 1) {
        out.x = R(0.5) * (Z.y + Zc.y);
        out.y = R(-0.5) * (Z.x - Zc.x);
      } else {
        out.x = R(0.5) * (Z.x + Zc.x);
        out.y = R(0.5) * (Z.y - Zc.y);
      }
      L.X[(size_t(ty * NL + mm) * NK + ki) * N + j0 + r_] = out;
    }
    __syncthreads();
  }
}

// y = S^(kappa)^+ x for the C values x_b = cur[b rs + kc], in place; the symbol entry e is
// S[e N + ks] (mixed form: from its deflated eigen form, FP64: the full block).
template <int K, bool MIXED>
__device__ __forceinline__ void symbol_product(const typename LatT<MIXED>::C2* S, int N, int ks,
                                               typename LatT<MIXED>::C2* cur, int rs, int kc) {
  using C2 = typename LatT<MIXED>::C2;
  constexpr int C = LatCtx<K, MIXED>::C;
  if constexpr (MIXED) {
    // y = v1 (v1^H x) / mu1 + R x, R the packed Hermitian remainder (R_ba = conj R_ab)
    C2 x[C], y[C];
    C2 s1 = {0, 0};
#pragma unroll
    for (int b = 0; b < C; ++b) {
      x[b] = cur[b * rs + kc];
      cmad_conj(s1, __ldg(&S[size_t(b) * N + ks]), x[b]);
    }
    const typename LatT<MIXED>::R d1 = __ldg(&S[size_t(C) * N + ks]).x;
    s1.x *= d1;
    s1.y *= d1;
#pragma unroll
    for (int a = 0; a < C; ++a) y[a] = cmul(__ldg(&S[size_t(a) * N + ks]), s1);
    int pi = C + 1;
#pragma unroll
    for (int a = 0; a < C; ++a)
#pragma unroll
      for (int b = a; b < C; ++b, ++pi) {
        const C2 h = __ldg(&S[size_t(pi) * N + ks]);
        cmad(y[a], h, x[b]);
        if (b != a) cmad_conj(y[b], h, x[a]);
      }
#pragma unroll
    for (int a = 0; a < C; ++a) cur[a * rs + kc] = y[a];
  } else {
    C2 x[C], y[C];
#pragma unroll
    for (int b = 0; b < C; ++b) {
      x[b] = cur[b * rs + kc];
      y[b] = C2{0, 0};
    }
#pragma unroll
    for (int a = 0; a < C; ++a)
#pragma unroll
      for (int b = 0; b < C; ++b) cmad(y[a], __ldg(&S[size_t(a * C + b) * N + ks]), x[b]);
#pragma unroll
    for (int a = 0; a < C; ++a) cur[a * rs + kc] = y[a];
  }
}

// Column pass: per ki, FFT along j, y = S^(kappa)^+ x, inverse FFT along j.
// Split form (L.split): the work items are (ki, parity p). With h = N/2 and w = exp(-2 pi i/N),
// one decimation-in-frequency step gives the even wavenumbers X[2k] = DFT_h(x_j + x_(j+h)) and
// the odd ones X[2k+1] = DFT_h((x_j - x_(j+h)) w^j); after the product, item p keeps the
// inverse half E = IDFT_h(Y_even) (p = 0) or w^-j IDFT_h(Y_odd) (p = 1) in X2, and the inverse
// row pass takes y_j = E_j + O_j, y_(j+h) = E_j - O_j. The symbol is stored with the even kj
// first, then the odd ones, so that each item reads a contiguous half.
template <int K, bool MIXED>
__device__ void columns(const LatCtx<K, MIXED>& L) {
  using C2 = typename LatT<MIXED>::C2;
  constexpr int C = LatCtx<K, MIXED>::C;
  constexpr int NP = LatCtx<K, MIXED>::NP;
  const int N = L.N, NK = L.NK;
  if (L.split) {
    const int h = N / 2;
    LatCtx<K, MIXED> Lh = L;
    Lh.N = h;
    Lh.logn = L.logn - 1;
    Lh.pow2 = (h & (h - 1)) == 0;
    Lh.tw = L.tw2;
    for (int item = blockIdx.x; item < 2 * NK; item += gridDim.x) {
      const int ki = item >> 1, par = item & 1;
#pragma unroll 6
      for (int e = threadIdx.x; e < C * h; e += blockDim.x) {
        const int c = e / h, j = e - c * h;
        const C2* col = &L.X[(size_t(c) * NK + ki) * N];
        const C2 a = __ldcg(&col[j]), b = __ldcg(&col[j + h]);
        L.bufa[e] = par ? cmul(csub(a, b), L.tw[j]) : cadd(a, b);
      }
      __syncthreads();
      xform(Lh, L.bufa, C, false);
      const C2* S = L.S + size_t(ki) * NP * N;
      for (int k = threadIdx.x; k < h; k += blockDim.x) symbol_product<K, MIXED>(S, N, par * h + k, L.bufa, h, k);
      __syncthreads();
      xform(Lh, L.bufa, C, true);
      for (int e = threadIdx.x; e < C * h; e += blockDim.x) {
        const int c = e / h, j = e - c * h;
        C2 v = L.bufa[e];
        if (par) {
          C2 w = L.tw[j];
          w.y = -w.y;
          v = cmul(v, w);
        }
        L.X2[(size_t(c) * NK + ki) * N + par * h + j] = v;
      }
      __syncthreads();
    }
    return;
  }
  for (int ki = blockIdx.x; ki < NK; ki += gridDim.x) {
#pragma unroll 12
    for (int e = threadIdx.x; e < C * N; e += blockDim.x) {
      const int c = e / N, j = e - c * N;
      L.bufa[e] = __ldcg(&L.X[(size_t(c) * NK + ki) * N + j]);
    }
    __syncthreads();
    xform(L, L.bufa, C, false);
    const C2* S = L.S + size_t(ki) * NP * N;
    for (int kj = threadIdx.x; kj < N; kj += blockDim.x) symbol_product<K, MIXED>(S, N, kj, L.bufa, N, kj);
    __syncthreads();
    xform(L, L.bufa, C, true);
    const C2* res = L.bufa;
    for (int e = threadIdx.x; e < C * N; e += blockDim.x) {
      const int c = e / N, j = e - c * N;
      L.X[(size_t(c) * NK + ki) * N + j] = res[e];
    }
    __syncthreads();
  }
}

// Row pass, inverse: rebuild W = Y_even + i Y_odd over all k (Y[N-k] = conj Y[k]),
// inverse FFT along i, z = the real / imaginary parts scaled by 1/N^2 in facet order.
// Accumulates r.z_new into rz and, if with_old, r.z_old into rzo.
template <int K, bool MIXED>
__device__ void rows_inverse(const LatCtx<K, MIXED>& L, bool with_old, typename LatT<MIXED>::Acc& rz,
                             typename LatT<MIXED>::Acc& rzo) {
  using T = LatT<MIXED>;
  using C2 = typename T::C2;
  using R = typename T::R;
  using Z = typename T::Z;
  constexpr int NL = K + 1, VS = LatCtx<K, MIXED>::VS;
  const int N = L.N, NK = L.NK;
  const R scale = R(1.0 / (double(N) * double(N)));
  const int ntiles = 3 * L.ntj;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ty = tile / L.ntj, j0 = (tile - ty * L.ntj) * kLatTJ;
    const int rows = min(kLatTJ, N - j0), npair = (rows + 1) >> 1;
#pragma unroll 8
    for (int e = threadIdx.x; e < npair * NK * NL; e += blockDim.x) {
      const int pr = e % npair, rest = e / npair;
      const int ki = rest % NK, mm = rest / NK;
      C2 ya, yb = C2{0, 0};
      if (L.split) {
        // y_j = E_j + O_j and y_(j+h) = E_j - O_j from the two halves of the split pass
        const int h = N >> 1;
        const C2* src = &L.X2[(size_t(ty * NL + mm) * NK + ki) * N];
        const int ja = j0 + 2 * pr, jb = ja + 1;
        const int ra = ja < h ? ja : ja - h, rb = jb < h ? jb : jb - h;
        const C2 ea = __ldcg(&src[ra]), oa = __ldcg(&src[h + ra]);
        ya = ja < h ? cadd(ea, oa) : csub(ea, oa);
        if (2 * pr + 1 < rows) {
          const C2 eb = __ldcg(&src[rb]), ob = __ldcg(&src[h + rb]);
          yb = jb < h ? cadd(eb, ob) : csub(eb, ob);
        }
      } else {
        const C2* src = &L.X[(size_t(ty * NL + mm) * NK + ki) * N + j0 + 2 * pr];
        ya = __ldcg(src);
        if (2 * pr + 1 < rows) yb = __ldcg(src + 1);
      }
      C2* w = L.bufa + (pr * NL + mm) * N;
      w[ki] = C2{ya.x - yb.y, ya.y + yb.x};
      if (ki > 0 && N - ki >= NK) w[N - ki] = C2{ya.x + yb.y, yb.x - ya.y};
    }
    __syncthreads();
    xform(L, L.bufa, npair * NL, true);
    const C2* res = L.bufa;
    const size_t base = (size_t(ty) * N + j0) * N * VS;
#pragma unroll 4
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
      const int r_ = e / N, i = e - r_ * N;
      const size_t o = base + size_t(e) * VS;
      typename T::A rv[NL];
      Z zv[NL], zo[NL];
      ldf<NL, VS>(L.r + o, rv);
      if (with_old) ldf<NL, VS>(L.z + o, zo);
#pragma unroll
      for (int mm = 0; mm < NL; ++mm) {
        const C2 v = res[((r_ >> 1) * NL + mm) * N + i];
        zv[mm] = Z((r_ & 1) ? v.y : v.x) * Z(scale);
        if (with_old) mad(rzo, rv[mm], zo[mm]);
        mad(rz, rv[mm], zv[mm]);
      }
      stf<NL, VS>(L.z + o, zv);
    }
    __syncthreads();
  }
}

// ---- loads of any vector type as the arithmetic type of its form
__device__ __forceinline__ double ldx(const double* p) { return __ldcg(p); }
__device__ __forceinline__ dfl ldx(const float2* p) { return to_dfl(__ldcg(p)); }
__device__ __forceinline__ float ldx(const float* p) { return __ldcg(p); }

// y = (S x)_f: the facet's own block and its four neighbours' (stencil class of f)
template <int NL, int VS, bool MIXED, typename X, typename XV>
__device__ __forceinline__ void spmv_lat(const DevMesh& m, int f, const X* x, XV, typename LatT<MIXED>::A (&y)[NL]) {
  using A = typename LatT<MIXED>::A;
  using Acc = typename LatT<MIXED>::Acc;
  int nb[5];
  facet_nbrs<NL>(m, f, nb);
  const size_t sb = size_t(__ldg(&m.facet_stencil[f])) * 5 * NL * NL;
  XV xs[5][NL];
#pragma unroll
  for (int b = 0; b < 5; ++b) ldf<NL, VS>(x + size_t(nb[b]) * VS, xs[b]);
  Acc acc[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) acc[i] = acc_zero(Acc{});
#pragma unroll
  for (int b = 0; b < 5; ++b)
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const XV xv = xs[b][j];
#pragma unroll
      for (int i = 0; i < NL; ++i) mad(acc[i], stencil_entry(m, sb + (b * NL + i) * NL + j, A{}), xv);
    }
#pragma unroll
  for (int i = 0; i < NL; ++i) y[i] = fin(acc[i]);
}

// The warm start of a solve from the multiplier history and its image under S in one pass:
// lam0 = c1 h1 + c2 h2 (h2 read only if use2) at facet f and at its four stencil neighbours,
// y = (S lam0)_f. Every facet forms its own and its neighbours' lam0 with the same operations,
// so lam0 (returned for f) is the same bits wherever it is formed.
template <int NL, int VS, bool MIXED>
__device__ __forceinline__ void spmv_lat_hist(const DevMesh& m, int f, const typename LatT<MIXED>::V* h1,
                                              const typename LatT<MIXED>::V* h2, typename LatT<MIXED>::A c1,
                                              typename LatT<MIXED>::A c2, bool use2,
                                              typename LatT<MIXED>::A (&lam0)[NL], typename LatT<MIXED>::A (&y)[NL]) {
  using A = typename LatT<MIXED>::A;
  using Acc = typename LatT<MIXED>::Acc;
  int nb[5];
  facet_nbrs<NL>(m, f, nb);
  const size_t sb = size_t(__ldg(&m.facet_stencil[f])) * 5 * NL * NL;
  A xs[5][NL];
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const size_t o = size_t(nb[b]) * VS;
    ldf<NL, VS>(h1 + o, xs[b]);
    if (use2) {
      A t[NL];
      ldf<NL, VS>(h2 + o, t);
#pragma unroll
      for (int j = 0; j < NL; ++j) xs[b][j] = c1 * xs[b][j] + c2 * t[j];
    } else {
#pragma unroll
      for (int j = 0; j < NL; ++j) xs[b][j] = c1 * xs[b][j];
    }
  }
  Acc acc[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) acc[i] = acc_zero(Acc{});
#pragma unroll
  for (int b = 0; b < 5; ++b)
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const A xv = xs[b][j];
#pragma unroll
      for (int i = 0; i < NL; ++i) mad(acc[i], stencil_entry(m, sb + (b * NL + i) * NL + j, A{}), xv);
    }
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    y[i] = fin(acc[i]);
    lam0[i] = xs[0][i];
  }
}

// g of facet f in the arithmetic type of the form
template <int NL>
__device__ __forceinline__ void facet_g(const DevMesh& m, int f, double (&gv)[NL]) {
  assemble_g<NL>(m, f, gv);
}
template <int NL>
__device__ __forceinline__ void facet_g(const DevMesh& m, int f, dfl (&gv)[NL]) {
  assemble_g_df<NL>(m, f, gv);
}

// ---- grid reductions of the per-thread partials, in the accumulator's own arithmetic
// (FP32 TwoSum pairs in the mixed form: no FP64 pipe): warps, then warp 0 for the block;
// the block partial goes to m.red (a dacc pair occupies the 8 bytes of a double slot);
// after the barrier every thread loads at most a couple of block partials, and the same
// warp / block steps give the grid sum, broadcast through shared memory. Fixed order:
// bitwise reproducible and identical in every block.
__device__ __forceinline__ double acc_combine(double a, double b) { return a + b; }
__device__ __forceinline__ dacc acc_combine(dacc a, dacc b) {
  float s, t;
  two_sum(a.s, b.s, s, t);
  return dacc{s, a.c + b.c + t};
}
__device__ __forceinline__ double shfl_acc(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dacc shfl_acc(dacc v, int o) {
  return dacc{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)};
}
template <typename Acc>
__device__ __forceinline__ Acc warp_acc(Acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = acc_combine(v, shfl_acc(v, o));
  return v;
}
__device__ __forceinline__ void red_store(double* p, double v) { *p = v; }
__device__ __forceinline__ void red_store(double* p, dacc v) { *reinterpret_cast<float2*>(p) = make_float2(v.s, v.c); }
__device__ __forceinline__ double red_load(const double* p, double) { return __ldcg(p); }
__device__ __forceinline__ dacc red_load(const double* p, dacc) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return dacc{v.x, v.y};
}

// Block sum of v in every thread (all threads of the block call it).
template <int N, typename Acc>
__device__ __forceinline__ void block_acc(Acc (&v)[N]) {
  __shared__ Acc part[kLatThreads / 32][N];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const Acc ws = warp_acc(v[i]);
    if (l == 0) part[w][i] = ws;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Acc b = (l < kLatThreads / 32) ? part[l][i] : acc_zero(Acc{});
    v[i] = warp_acc(b);
  }
  __syncthreads();
}

template <int N, typename Acc>
__device__ bool lat_reduce(const DevMesh& m, int slot0, const Acc (&v)[N], GridBar* bar, double (&out)[N]) {
  Acc b[N];
#pragma unroll
  for (int i = 0; i < N; ++i) b[i] = v[i];
  block_acc<N>(b);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < N; ++i) red_store(&m.red[size_t(slot0 + i) * kMaxSolverBlocks + blockIdx.x], b[i]);
  if (!grid_sync(bar, m.stats)) return false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Acc gsum = acc_zero(Acc{});
    for (int k = threadIdx.x; k < gridDim.x; k += blockDim.x)
      gsum = acc_combine(gsum, red_load(&m.red[size_t(slot0 + i) * kMaxSolverBlocks + k], Acc{}));
    b[i] = gsum;
  }
  block_acc<N>(b);
#pragma unroll
  for (int i = 0; i < N; ++i) out[i] = acc_val(b[i]);
  return true;
}

// Scalars of one PCG step, computed by thread 0 of each block (identically in every
// block) and broadcast through shared memory.
template <typename A>
struct LatScal {
  A alpha, alpha_lam, beta;
  int done, conv;
  double relres;
};

template <int K, bool MIXED>
__global__ void __launch_bounds__(kLatThreads, 2) k_solve_lat(DevMesh m, SolveArgs a) {
  using T = LatT<MIXED>;
  using C2 = typename T::C2;
  using R = typename T::R;
  using V = typename T::V;
  using A = typename T::A;
  using Acc = typename T::Acc;
  using Z = typename T::Z;
  constexpr int NL = K + 1, VS = LatCtx<K, MIXED>::VS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ LatScal<A> sc;
  LatCtx<K, MIXED> L;
  L.N = m.lat_N;
  L.logn = m.lat_logn;
  L.NK = L.N / 2 + 1;
  L.ntj = (L.N + kLatTJ - 1) / kLatTJ;
  L.pow2 = (L.N & (L.N - 1)) == 0;
  L.grp = m.lat_grp;
  L.tw = reinterpret_cast<C2*>(smem_raw);
  L.bufa = L.tw + L.N;
  L.scr = L.bufa + m.lat_bufsz;
  L.X = reinterpret_cast<C2*>(m.lat_x);
  L.S = reinterpret_cast<const C2*>(m.lat_sinv);
  L.split = m.lat_split != 0;
  L.tw2 = reinterpret_cast<C2*>(smem_raw) + m.lat_tw2_off;
  L.X2 = reinterpret_cast<C2*>(m.lat_x2);
  V* p;
  if constexpr (MIXED) {
    L.lam = m.lam_df;
    L.g = m.lv_g;
    L.r = m.lv_r;
    L.q = m.lv_q;
    L.z = m.lv_z;
    p = m.lv_p;
  } else {
    L.lam = m.lam;
    L.g = m.g;
    L.r = m.r;
    L.q = m.q;
    L.z = m.z;
    p = m.pa;
  }
  for (int t = threadIdx.x; t < L.N; t += blockDim.x) L.tw[t] = C2{R(m.lat_tw[2 * t]), R(m.lat_tw[2 * t + 1])};
  if (L.split)
    for (int t = threadIdx.x; t < L.N / 2; t += blockDim.x)
      L.tw2[t] = C2{R(m.lat_tw[4 * t]), R(m.lat_tw[4 * t + 1])};
  __syncthreads();
  const int nF = m.n_facet;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  GridBar* bar = m.bar;
  // g from both sides of every facet and the warm start lam0. With a history (the same stage
  // of earlier steps), lam0 = c1 hist1 + c2 hist2 and r = g - S lam0 in the same pass (every
  // facet forms its neighbours' lam0 from the history, which this launch only reads until
  // the first row pass moves it down one slot); otherwise lam0 = warm_scale lam (or zero),
  // and r = g - S lam0 takes a pass of its own after a grid barrier.
  const A warm = A(a.warm_scale), hc1 = A(a.c1), hc2 = A(a.c2);
  V* hist1 = static_cast<V*>(a.hist1);
  V* hist2 = static_cast<V*>(a.hist2);
  const bool use2 = a.c2 != 0.0;
  double ga = 0.0;
  Acc g0 = acc_zero(Acc{});
#pragma unroll 4
  for (int f = gtid; f < nF; f += gsz) {
    const size_t o = size_t(f) * VS;
    A gv[NL], lv[NL];
    facet_g<NL>(m, f, gv);
    if (hist1) {
      A y[NL];
      spmv_lat_hist<NL, VS, MIXED>(m, f, hist1, hist2, hc1, hc2, use2, lv, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) y[j] = gv[j] - y[j];
      stf<NL, VS>(L.r + o, y);
    } else {
      if (a.warm_scale != 0.0) {
        ldf<NL, VS>(L.lam + o, lv);
#pragma unroll
        for (int j = 0; j < NL; ++j) lv[j] = warm * lv[j];
      } else {
#pragma unroll
        for (int j = 0; j < NL; ++j) lv[j] = A(0);
      }
      stf<NL, VS>(L.g + o, gv);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const double lead = lead_d(gv[j]);
      ga = fma(lead, lead, ga);
    }
    stf<NL, VS>(L.lam + o, lv);
    acc_add(g0, gv[0]);
  }
  double gg[2];
  {
    const double gv2[2] = {ga, acc_val(g0)};
    if (!lat_reduce<2>(m, 4, gv2, bar, gg)) return;
  }
  const double c0 = gg[1] / double(nF);
  const double gnorm0 = sqrt(fmax(gg[0] - gg[1] * gg[1] / double(nF), 0.0));
  // PCG runs on the system scaled by sigma = 2^-e, e the exponent of the RMS entry of g
  // (exact in any precision): residuals and dot products stay near 1 whatever the size
  // of g, away from the FP32 exponent limits of the double-float form. r and p are
  // scaled, lam is not: lam += (alpha / sigma) p.
  const double sigma = gnorm0 > 0.0 ? ldexp(1.0, -ilogb(gnorm0 / sqrt(double(nF) * NL))) : 1.0;
  const double gnorm = sigma * gnorm0;
  const double stop2 = (a.rtol * gnorm) * (a.rtol * gnorm);
  // rounding floor: the recursive residual stops decreasing near eps * cond(S) relative
  // (double-float vectors: 1e-14..1e-12 on large meshes; FP64: near 1e-13 at N = 1024);
  // once an iteration no longer halves the residual and it is below floor_rtol, the
  // solve is accepted there
  const double floor2 = (a.floor_rtol * gnorm) * (a.floor_rtol * gnorm);
  int it = 0;
  bool conv = false;
  double relres = 0.0;
  if (gnorm == 0.0) {
    for (int f = gtid; f < nF; f += gsz) {
      const size_t o = size_t(f) * VS;
      A zero[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) zero[j] = A(0);
      stf<NL, VS>(L.lam + o, zero);
      if (hist1) {
        A hv[NL];
        ldf<NL, VS>(hist1 + o, hv);
        stf<NL, VS>(hist2 + o, hv);
      }
    }
    conv = true;
  } else {
    if (!hist1) {
      // r = g - S lam0
#pragma unroll 4
      for (int f = gtid; f < nF; f += gsz) {
        const size_t o = size_t(f) * VS;
        A y[NL], gv[NL];
        spmv_lat<NL, VS, MIXED>(m, f, L.lam, A{}, y);
        ldf<NL, VS>(L.g + o, gv);
#pragma unroll
        for (int j = 0; j < NL; ++j) y[j] = gv[j] - y[j];
        stf<NL, VS>(L.r + o, y);
      }
      if (!grid_sync(bar, m.stats)) return;
    }
    // z = M r
    // The constant multiplier is in the kernel of S and of the preconditioner, so PCG cannot
    // reduce r's component along it; rounding in every update adds to it (relative size
    // eps times the cancellation in S q). It is measured with r.r (the sum of the mode-0
    // entries), left out of the convergence test, and subtracted from r in the next update.
    // The first row pass scales r by sigma and removes the constant component of g from it:
    // r = sigma (g - c0 1 - S lam0).
    Acc rra[2] = {acc_zero(Acc{}), acc_zero(Acc{})};
    rows_forward<K, MIXED>(L, false, A(0), A(0), A(c0), p, rra[0], rra[1], A(sigma), hist1, hist2);
    double rr[2];
    if (!lat_reduce<2>(m, 6, rra, bar, rr)) return;
    double cmode = rr[1] / double(nF);
    rr[0] = fmax(rr[0] - rr[1] * rr[1] / double(nF), 0.0);
    columns<K, MIXED>(L);
    if (!grid_sync(bar, m.stats)) return;
    Acc rza[2] = {acc_zero(Acc{}), acc_zero(Acc{})};
    rows_inverse<K, MIXED>(L, false, rza[0], rza[1]);
    double rz[2];
    {
      const Acc rz1[1] = {rza[0]};
      double rzt[1];
      if (!lat_reduce<1>(m, 1, rz1, bar, rzt)) return;
      rz[0] = rzt[0];
    }
    double rho = rz[0], rrv = rr[0];
    double beta = 0.0;
    for (;; ++it) {
      // convergence and the scalars of this step, once per block
      if (threadIdx.x == 0) {
        sc.done = 0;
        sc.conv = 0;
        sc.relres = sqrt(rrv) / gnorm;
        if (!isfinite(rrv) || !isfinite(rho)) {
          if (blockIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
          sc.done = 1;
        } else if (rrv <= stop2) {
          sc.done = sc.conv = 1;
        } else if (it >= a.maxit) {
          sc.done = 1;
        }
        sc.beta = A(beta);
      }
      __syncthreads();
      relres = sc.relres;
      if (sc.done) {
        conv = sc.conv != 0;
        break;
      }
      // p = z + beta p, q = S p = S z + beta q (each facet updates only its own entries)
      const A bt = sc.beta;
      Acc pqa[1] = {acc_zero(Acc{})};
#pragma unroll 4
      for (int f = gtid; f < nF; f += gsz) {
        const size_t o = size_t(f) * VS;
        A y[NL], pv[NL], qv[NL];
        Z zz[NL];
        spmv_lat<NL, VS, MIXED>(m, f, L.z, Z{}, y);
        ldf<NL, VS>(L.z + o, zz);
        if (it > 0) {
          ldf<NL, VS>(p + o, pv);
          ldf<NL, VS>(L.q + o, qv);
        }
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const A zv = as_a(zz[j]);
          pv[j] = (it == 0) ? zv : zv + bt * pv[j];
          qv[j] = (it == 0) ? y[j] : y[j] + bt * qv[j];
          mad(pqa[0], pv[j], qv[j]);
        }
        stf<NL, VS>(p + o, pv);
        stf<NL, VS>(L.q + o, qv);
      }
      double pq[1];
      if (!lat_reduce<1>(m, 0, pqa, bar, pq)) return;
      if (threadIdx.x == 0) {
        sc.done = 0;
        if (!(pq[0] > 0.0)) {
          if (!isfinite(pq[0]) && blockIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
          sc.done = 1;
        } else {
          const double alpha = rho / pq[0];
          sc.alpha = A(alpha);
          sc.alpha_lam = A(alpha / sigma);
        }
      }
      __syncthreads();
      if (sc.done) break;
      // r -= alpha q, lam += alpha p, and the forward row pass of z = M r
      rra[0] = acc_zero(Acc{});
      rra[1] = acc_zero(Acc{});
      rows_forward<K, MIXED>(L, true, sc.alpha, sc.alpha_lam, A(cmode), p, rra[0], rra[1], A(1), nullptr, nullptr);
      if (!lat_reduce<2>(m, 6, rra, bar, rr)) return;
      cmode = rr[1] / double(nF);
      const double rr_prev = rrv;
      rrv = fmax(rr[0] - rr[1] * rr[1] / double(nF), 0.0);
      if (threadIdx.x == 0) {
        sc.done = 0;
        sc.conv = 0;
        const bool stagnated = rrv <= floor2 && rrv > 0.25 * rr_prev;
        if (rrv <= stop2 || !isfinite(rrv) || stagnated) {
          sc.done = 1;
          sc.relres = sqrt(rrv) / gnorm;
          sc.conv = isfinite(rrv) ? 1 : 0;
          if (!sc.conv && blockIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        }
      }
      __syncthreads();
      if (sc.done) {
        ++it;
        relres = sc.relres;
        conv = sc.conv != 0;
        break;
      }
      columns<K, MIXED>(L);
      if (!grid_sync(bar, m.stats)) return;
      rza[0] = acc_zero(Acc{});
      rza[1] = acc_zero(Acc{});
      rows_inverse<K, MIXED>(L, true, rza[0], rza[1]);
      if (!lat_reduce<2>(m, 1, rza, bar, rz)) return;
      // flexible (Polak-Ribiere) beta: the FP32 preconditioner is symmetric only up to rounding
      beta = (rz[0] - rz[1]) / rho;
      rho = rz[0];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats* st = m.stats;
    st->last_iters = it;
    st->total_iters += it;
    st->solves += 1;
    st->last_relres = relres;
    st->last_sweeps = 1;
    st->total_sweeps += 1;
    if (!conv) atomicOr(&st->flags, kFlagNotConverged);
  }
}

}  // namespace
}  // namespace dgdf
