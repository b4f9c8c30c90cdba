// K0: FP64 phase and twiddle tables.
//
// Also the two tables of the any-length DFTs (bluestein.cuh): the chirp W_{2N}^{j^2} and the
// spectrum of its conjugate, computed with an FP64 radix-2 FFT and rounded to float once.
//
// The rotate factor W_N^{(m2 m1') mod N} of the decomposed FFT (Eq. Chap4_2DFFT) and the
// Stockham pass twiddles are all of the form W_M^j with an exact integer j in [0, M) (the
// channelisers' down-conversion phases need no table: they are folded into the FFT's input
// order).  Each entry is computed once with FP64
// sincospi(2 j / M) (argument exact: M is a power of two) and rounded to float32, so no
// phase ever loses accuracy to an FP32 angle, even at M = 2^20.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_bf16.h>

#include "fft_tc.cuh"
#include "internal.h"

namespace scd {
namespace {

// Entries of the concatenated pass-twiddle table of a plan with radices (r0, r1, r2) (layout
// in PlanInfo, fft.cuh; r1 = 0: single pass, no table): the one length that the allocation and
// the kernel that fills it both use.
__host__ __device__ constexpr int pass_table_len(int r0, int r1, int r2) {
  return r1 == 0 ? 0 : r0 * r1 + (r2 ? r0 * r1 * r2 : 0);
}

__device__ __forceinline__ float2 root_fp64(int64_t j, int64_t M) {
  double s, c;
  sincospi(2.0 * (double)j / (double)M, &s, &c);
  return make_float2((float)c, (float)(-s));
}

__global__ void k_roots(float2* out, int64_t M) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = root_fp64(j, M);
}

// Stockham pass twiddles: for pass s (s >= 1) with p = prod of earlier radices and radix R,
// entry off_s + r p + k = W_{pR}^{k r} = W_M^{k r M/(pR)} (k < p, r < R, so the index is < M).
__global__ void k_pass(float2* out, int M, int r0, int r1, int r2) {
  const int total = pass_table_len(r0, r1, r2);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x)
    out[e] = root_fp64(pass_twiddle_exponent(e, M, r0, r1, r2), M);
}

// W_N^{c m1'} for c < C, m1' < M1 at [m1'][c] (c m1' < C M1 <= N: no reduction needed)
__global__ void k_cols(float2* out, int64_t N, int M1, int C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M1 * C; e += gridDim.x * blockDim.x) {
    const int m1 = e / C, c = e % C;
    out[e] = root_fp64(((int64_t)c * m1) % N, N);
  }
}

// Complex-as-real DFT matrix of radix R for the tensor-core form, as bf16 hi and lo in the
// canonical K-major layout (N = K = Kp rows/columns, zero beyond 2R):
//   B[2j][2r] = B[2j+1][2r+1] = Re W_R^{jr},  B[2j][2r+1] = -Im W_R^{jr},  B[2j+1][2r] = Im W_R^{jr}
// so that [Yr Yi] = [Xr Xi] B^T computes Y_j = sum_r X_r W_R^{jr}.
__global__ void k_dftmat(unsigned char* out, int R, int Kp) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Kp * Kp; e += gridDim.x * blockDim.x) {
    const int n = e / Kp, k = e % Kp;
    double v = 0.0;
    if (n < 2 * R && k < 2 * R) {
      const int j = n >> 1, r = k >> 1;
      double s, c;
      sincospi(2.0 * (double)((j * r) % R) / (double)R, &s, &c);
      const double wr = c, wi = -s;
      v = (n & 1) == 0 ? ((k & 1) == 0 ? wr : -wi) : ((k & 1) == 0 ? wi : wr);
    }
    const __nv_bfloat16 hi = __double2bfloat16(v);
    const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
    const uint32_t off = umma::kmajor_offset(n, k, Kp);
    *reinterpret_cast<__nv_bfloat16*>(out + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(out + Kp * Kp * 2 + off) = lo;
  }
}

__global__ void k_hamming(float* out, int Np) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < Np) out[n] = (float)(0.54 - 0.46 * cospi(2.0 * (double)n / (double)(Np - 1)));
}

// Dolph-Chebyshev window (the `chebwin` of Algorithms 1 and 2), one block of Np <= 256
// threads, FP64 throughout: spectrum samples W(k) = T_{Np-1}(x0 cos(pi k / Np)) with
// x0 = cosh(acosh(10^{A/20}) / (Np - 1)); the window symmetric about (Np - 1)/2 is the real
// cosine sum w[n] = W(0) + 2 sum_{k=1}^{floor((Np-1)/2)} W(k) cos(pi k (2n - Np + 1) / Np),
// scaled to a peak of 1 and rounded to float32 once.
__device__ double chebyshev_poly(int M, double x) {
  if (fabs(x) <= 1.0) return cos(M * acos(x));
  const double v = cosh(M * acosh(fabs(x)));
  return (x < 0.0 && (M & 1)) ? -v : v;
}

__global__ void __launch_bounds__(256) k_chebwin(float* out, int Np, double atten_db) {
  __shared__ double red[256];
  const int n = threadIdx.x, M = Np - 1;
  const double x0 = cosh(acosh(pow(10.0, atten_db / 20.0)) / M);
  double v = 0.0;
  if (n < Np) {
    v = chebyshev_poly(M, x0);
    for (int k = 1; k <= (Np - 1) / 2; ++k)
      v += 2.0 * chebyshev_poly(M, x0 * cospi((double)k / Np)) * cospi((double)(k * (2 * n - Np + 1)) / Np);
  }
  red[n] = n < Np ? v : -1.0e300;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (n < s) red[n] = fmax(red[n], red[n + s]);
    __syncthreads();
  }
  if (n < Np) out[n] = (float)(v / red[0]);
}

// Chirp of Bluestein's identity for a length-N DFT: c[j] = W_{2N}^{(j^2) mod 2N}, j < N (the
// exponent reduced exactly in 64-bit integers before it becomes an angle).
__global__ void k_chirp(float2* out, int64_t N) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = root_fp64((j * j) % (2 * N), 2 * N);
}

// bt[j] = conj(c[j]) for j < N, conj(c[M - j]) for M - j < N, 0 between (FP64).
__global__ void k_bluestein_kernel(double2* bt, int64_t N, int64_t M) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = j < N ? j : (M - j < N ? M - j : -1);
    double s = 0.0, c = 0.0;
    if (i >= 0) sincospi((double)((i * i) % (2 * N)) / (double)N, &s, &c);
    bt[j] = i >= 0 ? make_double2(c, s) : make_double2(0.0, 0.0);       // conj(W_{2N}^{i^2})
  }
}

// One radix-2 pass of an FP64 Stockham FFT of size M (the recurrence of fft.cuh with R = 2):
// for s < M/(2p), k < p:  a = in[k + s p], b = in[k + (s + M/(2p)) p] W_{2p}^k,
// out[k + 2 s p] = a + b, out[k + p + 2 s p] = a - b.  After the pass with p = M/2 the output is
// the transform in natural order.
__global__ void k_fft64_pass(const double2* __restrict__ in, double2* __restrict__ out, int64_t M, int64_t p) {
  const int64_t half = M / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < half; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / p, k = e % p;
    double sn, cs;
    sincospi((double)k / (double)p, &sn, &cs);
    const double2 a = in[k + s * p], bi = in[k + (s + half / p) * p];
    const double2 b = make_double2(bi.x * cs + bi.y * sn, bi.y * cs - bi.x * sn);   // bi W_{2p}^k
    out[k + 2 * s * p] = make_double2(a.x + b.x, a.y + b.y);
    out[k + p + 2 * s * p] = make_double2(a.x - b.x, a.y - b.y);
  }
}

__global__ void k_scale_round(const double2* __restrict__ in, float2* __restrict__ out, int64_t M) {
  const double inv = 1.0 / (double)M;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = make_float2((float)(in[j].x * inv), (float)(in[j].y * inv));
}

// Row-major copy of the kernel spectrum for the fused middle pass of the any-N strip transform:
// out[q1 M2 + q2] = bh[q1 + M1 q2] (a permutation of float values, exact).
__global__ void k_permute_rows(const float2* __restrict__ bh, float2* __restrict__ out, int64_t M, int64_t M1) {
  const int64_t M2 = M / M1;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = bh[j / M2 + M1 * (j % M2)];
}

struct Key {
  int dev, kind;
  int64_t a, b, c;
  bool operator<(const Key& o) const { return std::tie(dev, kind, a, b, c) < std::tie(o.dev, o.kind, o.a, o.b, o.c); }
};

std::mutex g_mu;
std::map<Key, void*> g_tables;

struct PassRadices { int r0, r1, r2; };
PassRadices pass_radices(int M) {
  PassRadices r{0, 0, 0};
#define SCD_PR(MM) r = {Plan<MM>::r[0], Plan<MM>::r[1], Plan<MM>::r[2]}
  switch (M) {
    case 2: SCD_PR(2); break;       case 4: SCD_PR(4); break;       case 8: SCD_PR(8); break;
    case 16: SCD_PR(16); break;     case 32: SCD_PR(32); break;     case 64: SCD_PR(64); break;
    case 128: SCD_PR(128); break;   case 256: SCD_PR(256); break;   case 512: SCD_PR(512); break;
    case 1024: SCD_PR(1024); break; case 2048: SCD_PR(2048); break; case 4096: SCD_PR(4096); break;
    case 8192: SCD_PR(8192); break; case 16384: SCD_PR(16384); break;
    default: break;
  }
#undef SCD_PR
  return r;
}

// Returns the cached table for key, building it with `build(ptr, stream)` on first use.
template <class Build>
void* get_or_build(int kind, int64_t a, int64_t b, int64_t c, size_t bytes, cudaError_t* err, Build build) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  Key key{dev, kind, a, b, c};
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_tables.find(key);
  if (it != g_tables.end()) return it->second;
  void* ptr = nullptr;
  if ((*err = cudaMalloc(&ptr, bytes)) != cudaSuccess) return nullptr;
  cudaStream_t st;
  if ((*err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { cudaFree(ptr); return nullptr; }
  build(ptr, st);
  *err = cudaGetLastError();
  if (*err == cudaSuccess) *err = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (*err != cudaSuccess) { cudaFree(ptr); return nullptr; }
  g_tables[key] = ptr;
  return ptr;
}

int grid_for(int64_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

const float2* table_roots(int M, cudaError_t* err) {
  return (const float2*)get_or_build(0, M, 0, 0, sizeof(float2) * (size_t)M, err, [&](void* p, cudaStream_t st) {
    k_roots<<<grid_for(M), 256, 0, st>>>((float2*)p, M);
  });
}

const float2* table_pass(int M, cudaError_t* err) {
  PassRadices r = pass_radices(M);
  if (r.r0 == 0) { *err = cudaErrorInvalidValue; return nullptr; }
  int len = r.r1 ? pass_table_len(r.r0, r.r1, r.r2) : 1;
  return (const float2*)get_or_build(1, M, 0, 0, sizeof(float2) * (size_t)len, err, [&](void* p, cudaStream_t st) {
    if (r.r1) k_pass<<<grid_for(len), 256, 0, st>>>((float2*)p, M, r.r0, r.r1, r.r2);
    else cudaMemsetAsync(p, 0, sizeof(float2), st);
  });
}

const float2* table_cols(int N, int M1, int C, cudaError_t* err) {
  return (const float2*)get_or_build(2, N, M1, C, sizeof(float2) * (size_t)M1 * C, err, [&](void* p, cudaStream_t st) {
    k_cols<<<grid_for((int64_t)M1 * C), 256, 0, st>>>((float2*)p, N, M1, C);
  });
}

const float2* table_chirp(int64_t N, cudaError_t* err) {
  return (const float2*)get_or_build(8, N, 0, 0, sizeof(float2) * (size_t)N, err, [&](void* p, cudaStream_t st) {
    k_chirp<<<grid_for(N), 256, 0, st>>>((float2*)p, N);
  });
}

const float2* table_bluestein(int64_t N, int64_t M, cudaError_t* err) {
  if (M < 2 * N - 1 || !is_pow2(M)) { *err = cudaErrorInvalidValue; return nullptr; }
  return (const float2*)get_or_build(9, N, M, 0, sizeof(float2) * (size_t)M, err, [&](void* p, cudaStream_t st) {
    double2* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, sizeof(double2) * 2 * (size_t)M, st) != cudaSuccess) return;
    double2* a = buf;
    double2* b = buf + M;
    k_bluestein_kernel<<<grid_for(M), 256, 0, st>>>(a, N, M);
    for (int64_t q = 1; q < M; q <<= 1) {
      k_fft64_pass<<<grid_for(M / 2), 256, 0, st>>>(a, b, M, q);
      double2* t = a; a = b; b = t;
    }
    k_scale_round<<<grid_for(M), 256, 0, st>>>(a, (float2*)p, M);
    cudaFreeAsync(buf, st);
  });
}

const float2* table_bluestein_rows(int64_t N, int64_t M, int M1, cudaError_t* err) {
  const float2* bh = table_bluestein(N, M, err);            // built first: get_or_build holds its lock
  if (!bh) return nullptr;
  if (M1 <= 0 || M % M1 != 0) { *err = cudaErrorInvalidValue; return nullptr; }
  return (const float2*)get_or_build(10, N, M, M1, sizeof(float2) * (size_t)M, err, [&](void* p, cudaStream_t st) {
    k_permute_rows<<<grid_for(M), 256, 0, st>>>(bh, (float2*)p, M, M1);
  });
}

const float* table_hamming(int Np, cudaError_t* err) {
  return (const float*)get_or_build(3, Np, 0, 0, sizeof(float) * (size_t)Np, err, [&](void* p, cudaStream_t st) {
    k_hamming<<<(Np + 255) / 256, 256, 0, st>>>((float*)p, Np);
  });
}

cudaError_t build_pass_into(float2* out, int M, cudaStream_t st) {
  PassRadices r = pass_radices(M);
  if (r.r0 == 0) return cudaErrorInvalidValue;
  if (!r.r1) return cudaSuccess;                               // single-pass plans use no table
  const int len = pass_table_len(r.r0, r.r1, r.r2);
  k_pass<<<grid_for(len), 256, 0, st>>>(out, M, r.r0, r.r1, r.r2);
  return cudaGetLastError();
}

cudaError_t build_chebyshev_into(float* out, int Np, double atten_db, cudaStream_t st) {
  k_chebwin<<<1, 256, 0, st>>>(out, Np, atten_db);
  return cudaGetLastError();
}

cudaError_t build_hamming_into(float* out, int Np, cudaStream_t st) {
  k_hamming<<<(Np + 255) / 256, 256, 0, st>>>(out, Np);
  return cudaGetLastError();
}

// B matrices of every distinct radix of the size-M plan, concatenated in slot order
// (the order TcPlan<M, *>::boff() expects).
const unsigned char* table_tc_bmats(int M, int* bytes, cudaError_t* err) {
  PassRadices r = pass_radices(M);
  if (r.r0 == 0) { *err = cudaErrorInvalidValue; return nullptr; }
  int radix[3] = {r.r0, r.r1, r.r2};
  int nslots = 1, slot_radix[3] = {r.r0, 0, 0};
  for (int s = 1; s < 3; ++s) {
    if (!radix[s]) break;
    bool seen = false;
    for (int q = 0; q < nslots; ++q) seen |= slot_radix[q] == radix[s];
    if (!seen) slot_radix[nslots++] = radix[s];
  }
  int total = 0, off[3];
  for (int q = 0; q < nslots; ++q) { off[q] = total; total += 2 * tc_bmat_bytes(slot_radix[q]); }
  *bytes = total;
  return (const unsigned char*)get_or_build(4, M, 0, 0, (size_t)total, err, [&](void* p, cudaStream_t st) {
    for (int q = 0; q < nslots; ++q) {
      const int Kp = tc_kp(slot_radix[q]);
      k_dftmat<<<grid_for((int64_t)Kp * Kp), 256, 0, st>>>((unsigned char*)p + off[q], slot_radix[q], Kp);
    }
  });
}

unsigned* device_error_word(cudaError_t* err) {
  return (unsigned*)get_or_build(5, 0, 0, 0, 16, err, [&](void* p, cudaStream_t st) {
    cudaMemsetAsync(p, 0, 16, st);
  });
}

void release_tables() {
  std::lock_guard<std::mutex> lock(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_tables) {
    cudaSetDevice(kv.first.dev);
    cudaFree(kv.second);
  }
  cudaSetDevice(cur);
  g_tables.clear();
}

}  // namespace scd
