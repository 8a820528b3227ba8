// Host side of the lattice facet solver (the kernel is in k_lattice_kernel.cuh): sizes of its
// shared-memory buffers and of the stored symbol, the launch shape and the launch. Each
// instantiation k_solve_lat<K, MIXED> lives in its own object file (k_lattice_inst.cu).
#include "k_lattice_kernel.cuh"

namespace dgdf {

// defined in k_lattice_inst.cu, one object file per (K, form)
const void* lattice_kernel_k1_0();
const void* lattice_kernel_k1_1();
const void* lattice_kernel_k2_0();
const void* lattice_kernel_k2_1();
const void* lattice_kernel_k3_0();
const void* lattice_kernel_k3_1();

namespace {

const void* lattice_kernel(int k, int fp32) {
  switch (k * 2 + (fp32 ? 1 : 0)) {
    case 2: return lattice_kernel_k1_0();
    case 3: return lattice_kernel_k1_1();
    case 4: return lattice_kernel_k2_0();
    case 5: return lattice_kernel_k2_1();
    case 6: return lattice_kernel_k3_0();
    case 7: return lattice_kernel_k3_1();
    default: return nullptr;
  }
}

}  // namespace

size_t lattice_buffer_elems(int k, int N, int fp32) {
  (void)fp32;
  const size_t C = 3 * (k + 1), rows_buf = size_t(k + 1) * (kLatTJ / 2);
  return (C > rows_buf ? C : rows_buf) * N;
}

// Scratch row: N, plus the padding of the two-pass FFT (R2 = 2^floor(log2 N / 2)).
size_t lattice_scratch_row(int N) {
  int logn = 0;
  while ((1 << logn) < N) ++logn;
  return (1 << logn) == N ? size_t(N) + (size_t(1) << (logn / 2)) : size_t(N);
}

// The split pays where the N/2+1 columns leave blocks idle: N even, N >= 64, and at most one
// column per SM (2 blocks per SM); at N = 1024 it was 3% slower per PCG iteration.
bool lattice_split(int N) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return N % 2 == 0 && N >= 64 && N / 2 + 1 <= sms;
}

size_t lattice_tw2_offset(int k, int N, int fp32, int grp) {
  return size_t(N) + lattice_buffer_elems(k, N, fp32) + size_t(grp) * lattice_scratch_row(N);
}

size_t lattice_smem_bytes(int k, int N, int fp32, int grp) {
  const size_t cx = fp32 ? 8 : 16;
  return (lattice_tw2_offset(k, N, fp32, grp) + (lattice_split(N) ? size_t(N / 2) : 0)) * cx;
}

// Rows per transform group: all of them if two blocks per SM still fit, else the most
// that fit at two blocks per SM, else at one block per SM; 0 if not even one row fits.
int lattice_group_rows(int k, int N, int fp32) {
  int dev = 0, optin = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int rows = int(lattice_buffer_elems(k, N, fp32) / size_t(N));
  const size_t two = size_t(per_sm) / 2 - 2048, one = size_t(optin) - 2048;
  for (size_t budget : {two, one})
    for (int g = rows; g >= 1; --g)
      if (lattice_smem_bytes(k, N, fp32, g) <= budget) return g;
  return 0;
}

size_t lattice_symbol_elems(int k, int N, int fp32) {
  const size_t C = 3 * (k + 1);
  return size_t(N / 2 + 1) * (fp32 ? C + 1 + C * (C + 1) / 2 : C * C) * N;
}

size_t lattice_spectrum_elems(int k, int N) { return size_t(3 * (k + 1)) * (N / 2 + 1) * N; }

int lattice_blocks(int k, int N, int fp32) {
  const void* fn = lattice_kernel(k, fp32);
  if (!fn) return 0;
  const int grp = lattice_group_rows(k, N, fp32);
  if (grp < 1) return 0;
  const size_t smem = lattice_smem_bytes(k, N, fp32, grp);
  int per_sm = 0, dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  // the attribute is per kernel, shared by all meshes: allow the device maximum once,
  // so that meshes of different sizes can use the same instantiation
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int max_dyn = optin - int(fa.sharedSizeBytes);
  if (max_dyn <= 0 || smem > size_t(max_dyn)) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLatThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm < 1) return 0;
  int nb = sms * (per_sm < 2 ? per_sm : 2);
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  return nb;
}

cudaError_t launch_solve_lattice(const DevMesh& m, const SolveArgs& a, int nblocks, int fp32, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  const void* fn = lattice_kernel(m.k, fp32);
  if (!fn) return cudaErrorInvalidValue;
  DevMesh mm = m;
  SolveArgs aa = a;
  void* args[] = {&mm, &aa};
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kLatThreads), args,
                                     lattice_smem_bytes(m.k, m.lat_N, fp32, m.lat_grp), s);
}

}  // namespace dgdf
