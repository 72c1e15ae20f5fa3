// CUDA kernels of the GB300 RIC-MRCCSD library (sm_103a, FP64 paths).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"
#include "kernels.h"

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Generic contraction C[l,m,n] += alpha * sum_k A[l,m,k] B[l,n,k]
// Index -> element offsets through per-group offset tables (see internal.h).
// ---------------------------------------------------------------------------
template <int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_contract_tile(const double* __restrict__ A, const double* __restrict__ B,
                    double* __restrict__ C, const int64_t* __restrict__ tab, int64_t L,
                    int64_t M, int64_t N, int64_t K, int ksplit, int64_t kchunk, double alpha) {
  constexpr int NT = (BM / TM) * (BN / TN);
  const int64_t* tAL = tab;
  const int64_t* tBL = tAL + L;
  const int64_t* tCL = tBL + L;
  const int64_t* tAM = tCL + L;
  const int64_t* tCM = tAM + M;
  const int64_t* tBN = tCM + M;
  const int64_t* tCN = tBN + N;
  const int64_t* tAK = tCN + N;
  const int64_t* tBK = tAK + K;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ int64_t sAM[BM], sCM[BM], sBN[BN], sCN[BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  const int64_t mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
  const int64_t ntile = L * ksplit * mt * nt;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    int64_t r = tile;
    const int64_t ni = r % nt;
    r /= nt;
    const int64_t mi = r % mt;
    r /= mt;
    const int ks = (int)(r % ksplit);
    const int64_t l = r / ksplit;
    const int64_t m0 = mi * BM, n0 = ni * BN;
    for (int i = tid; i < BM; i += NT) {
      const int64_t m = m0 + i;
      sAM[i] = m < M ? tAM[m] : 0;
      sCM[i] = m < M ? tCM[m] : 0;
    }
    for (int i = tid; i < BN; i += NT) {
      const int64_t n = n0 + i;
      sBN[i] = n < N ? tBN[n] : 0;
      sCN[i] = n < N ? tCN[n] : 0;
    }
    const int64_t aL = tAL[l], bL = tBL[l], cL = tCL[l];
    const int64_t kb = (int64_t)ks * kchunk;
    const int64_t ke = kb + kchunk < K ? kb + kchunk : K;
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
      for (int i = tid; i < BK * BM; i += NT) {
        const int kk = i / BM, mm = i % BM;
        const int64_t k = k0 + kk, m = m0 + mm;
        As[kk][mm] = (k < ke && m < M) ? A[aL + sAM[mm] + tAK[k]] : 0.0;
      }
      for (int i = tid; i < BK * BN; i += NT) {
        const int kk = i / BN, nn = i % BN;
        const int64_t k = k0 + kk, n = n0 + nn;
        Bs[kk][nn] = (k < ke && n < N) ? B[bL + sBN[nn] + tBK[k]] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        double a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int mm = ty * TM + i;
      if (m0 + mm >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int nn = tx * TN + j;
        if (n0 + nn >= N) continue;
        if (acc[i][j] != 0.0) atomicAdd(C + cL + sCM[mm] + sCN[nn], alpha * acc[i][j]);
      }
    }
    __syncthreads();
  }
}

__device__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads)
    k_contract_dot(const double* __restrict__ A, const double* __restrict__ B,
                   double* __restrict__ C, const int64_t* __restrict__ tab, int64_t L,
                   int64_t M, int64_t N, int64_t K, int ksplit, int64_t kchunk, double alpha) {
  const int64_t* tAL = tab;
  const int64_t* tBL = tAL + L;
  const int64_t* tCL = tBL + L;
  const int64_t* tAM = tCL + L;
  const int64_t* tCM = tAM + M;
  const int64_t* tBN = tCM + M;
  const int64_t* tCN = tBN + N;
  const int64_t* tAK = tCN + N;
  const int64_t* tBK = tAK + K;
  const int64_t nwork = L * M * N * ksplit;
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int ks = (int)(w % ksplit);
    const int64_t o = w / ksplit;
    const int64_t l = o / (M * N), mn = o % (M * N), m = mn / N, n = mn % N;
    const int64_t ao = tAL[l] + tAM[m], bo = tBL[l] + tBN[n];
    const int64_t kb = (int64_t)ks * kchunk;
    const int64_t ke = kb + kchunk < K ? kb + kchunk : K;
    double s = 0.0;
    for (int64_t k = kb + threadIdx.x; k < ke; k += blockDim.x) s = fma(A[ao + tAK[k]], B[bo + tBK[k]], s);
    s = block_sum(s);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(C + tCL[l] + tCM[m] + tCN[n], alpha * s);
  }
}

__global__ void k_fill(double* p, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void launch_contract(const ContractOp& op, const int64_t* d_table, cudaStream_t s) {
  if (op.L == 0 || op.M == 0 || op.N == 0 || op.K == 0) return;
  const int64_t* tab = d_table + op.tab;
  if (op.kind == 2) {
    int64_t work = op.L * op.M * op.N * op.ksplit;
    int g = (int)(work < 152 * 16 ? work : 152 * 16);
    k_contract_dot<<<g, kThreads, 0, s>>>(op.A, op.B, op.C, tab, op.L, op.M, op.N, op.K, op.ksplit,
                                          op.kchunk, op.alpha);
  } else if (op.kind == 0) {
    int64_t tiles = op.L * op.ksplit * ((op.M + 63) / 64) * ((op.N + 63) / 64);
    int g = (int)(tiles < 152 * 8 ? tiles : 152 * 8);
    k_contract_tile<64, 64, 4, 4, 16><<<g, 256, 0, s>>>(op.A, op.B, op.C, tab, op.L, op.M, op.N,
                                                         op.K, op.ksplit, op.kchunk, op.alpha);
  } else {
    int64_t tiles = op.L * op.ksplit * ((op.M + 15) / 16) * ((op.N + 15) / 16);
    int g = (int)(tiles < 152 * 16 ? tiles : 152 * 16);
    k_contract_tile<16, 16, 1, 1, 16><<<g, 256, 0, s>>>(op.A, op.B, op.C, tab, op.L, op.M, op.N,
                                                         op.K, op.ksplit, op.kchunk, op.alpha);
  }
}

void launch_fill(double* p, double v, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<<<grid_for(n), kThreads, 0, s>>>(p, v, n);
}

// ---------------------------------------------------------------------------
// Amplitude packing: flat class layout <-> general particle/hole tensors
// ---------------------------------------------------------------------------
namespace {
__global__ void k_scatter(double* __restrict__ dst, const double* __restrict__ src,
                          const int64_t* __restrict__ idx, const int64_t* __restrict__ idx2,
                          int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[i];
    dst[idx[i]] = x;
    if (idx2 != nullptr && idx2[i] >= 0) dst[idx2[i]] = x;
  }
}
__global__ void k_gather(double* __restrict__ dst, const double* __restrict__ src,
                         const int64_t* __restrict__ idx, const int64_t* __restrict__ idx2, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]] + (idx2 != nullptr ? src[idx2[i]] : 0.0);
}
}  // namespace

void launch_scatter(double* dst, const double* src, const int64_t* idx, const int64_t* idx2,
                    int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_scatter<<<grid_for(n), kThreads, 0, s>>>(dst, src, idx, idx2, n);
}
void launch_gather(double* dst, const double* src, const int64_t* idx, const int64_t* idx2,
                   int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_gather<<<grid_for(n), kThreads, 0, s>>>(dst, src, idx, idx2, n);
}

// ---------------------------------------------------------------------------
// Reference quantities (Sec. 2.1) in spin-free form
// ---------------------------------------------------------------------------
namespace {
// f_pq = h_pq + sum_m [2 (pq|mm) - (pm|mq)] + sum_tu G1_tu [(pq|tu) - 1/2 (pu|tq)]
__global__ void k_fock(double* __restrict__ F, const double* __restrict__ h,
                       const double* __restrict__ eri, const double* __restrict__ g1, Dims d) {
  const int64_t n = d.n, n2 = n * n, n3 = n2 * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / n, q = i % n;
    double f = h[i];
    for (int m = 0; m < d.o; ++m) f += 2.0 * eri[p * n3 + q * n2 + m * n + m] - eri[p * n3 + m * n2 + m * n + q];
    for (int t = 0; t < d.a; ++t)
      for (int u = 0; u < d.a; ++u) {
        const int64_t T = d.o + t, U = d.o + u;
        f += g1[t * d.a + u] * (eri[p * n3 + q * n2 + T * n + U] - 0.5 * eri[p * n3 + U * n2 + T * n + q]);
      }
    F[i] = f;
  }
}

// E0 = 1/2 sum_{pq in H} D_pq (h_pq + f_pq) + 1/2 sum_{tuvw} (tu|vw) L2[t,v,u,w]
__global__ void k_e0(double* __restrict__ out, const double* __restrict__ h,
                     const double* __restrict__ F, const double* __restrict__ eri,
                     const double* __restrict__ g1, const double* __restrict__ l2, Dims d) {
  const int64_t n = d.n, n2 = n * n, n3 = n2 * n;
  const int64_t a = d.a, a2 = a * a, a3 = a2 * a;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < (int64_t)d.o; i += blockDim.x) s += (h[i * n + i] + F[i * n + i]);
  for (int64_t i = threadIdx.x; i < a2; i += blockDim.x) {
    const int64_t t = i / a, u = i % a, T = d.o + t, U = d.o + u;
    s += 0.5 * g1[i] * (h[T * n + U] + F[T * n + U]);
  }
  for (int64_t i = threadIdx.x; i < a2 * a2; i += blockDim.x) {
    const int64_t t = i / a3, u = (i / a2) % a, v = (i / a) % a, w = i % a;
    const int64_t T = d.o + t, U = d.o + u, V = d.o + v, W = d.o + w;
    s += 0.5 * eri[T * n3 + U * n2 + V * n + W] * l2[t * a3 + v * a2 + u * a + w];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// Lambda2 = Gamma2 - G1 G1 + 1/2 G1 G1 (exchange); D2 = (2 L2 + L2^{qp}_{rs}) / 6;
// G = G1/2, E = 1 - G.
__global__ void k_cumulant2(double* __restrict__ L2, double* __restrict__ D2, double* __restrict__ G,
                            double* __restrict__ E, const double* __restrict__ g1,
                            const double* __restrict__ g2, int a, int given_cumulant) {
  const int64_t a2 = (int64_t)a * a, a3 = a2 * a, a4 = a2 * a2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a4; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / a3, q = (i / a2) % a, r = (i / a) % a, s = i % a;
    double l = g2[i];
    if (!given_cumulant) l += -g1[p * a + r] * g1[q * a + s] + 0.5 * g1[p * a + s] * g1[q * a + r];
    L2[i] = l;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a2; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / a, q = i % a;
    G[i] = 0.5 * g1[i];
    E[i] = (p == q ? 1.0 : 0.0) - 0.5 * g1[i];
  }
}
__global__ void k_direct2(double* __restrict__ D2, const double* __restrict__ L2, int a) {
  const int64_t a2 = (int64_t)a * a, a3 = a2 * a, a4 = a2 * a2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a4; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / a3, q = (i / a2) % a, rs = i % a2;
    D2[i] = (2.0 * L2[i] + L2[q * a3 + p * a2 + rs]) / 6.0;
  }
}
// D3 = W L3 with W = (17 e - sum transpositions - 7 sum 3-cycles) / 144 acting on
// the lower indices: the pseudo-inverse of sum_pi sgn(pi) 2^{cycles(pi)} pi.
__global__ void k_direct3(double* __restrict__ D3, const double* __restrict__ L3, int a) {
  const int64_t a1 = a, a2 = a1 * a1, a3 = a2 * a1;
  const int64_t tot = a3 * a3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t up = i / a3;
    const int64_t s = (i / a2) % a1, t = (i / a1) % a1, u = i % a1;
    const double* b = L3 + up * a3;
#define LW(x, y, z) b[(x) * a2 + (y) * a1 + (z)]
    const double v = 17.0 * LW(s, t, u) - LW(t, s, u) - LW(u, t, s) - LW(s, u, t) -
                     7.0 * LW(t, u, s) - 7.0 * LW(u, s, t);
#undef LW
    D3[i] = v / 144.0;
  }
}
}  // namespace

void launch_fock(double* F, const double* h, const double* eri, const double* g1, const Dims& d,
                 cudaStream_t s) {
  k_fock<<<grid_for((int64_t)d.n * d.n), kThreads, 0, s>>>(F, h, eri, g1, d);
}
void launch_e0(double* out, const double* h, const double* F, const double* eri, const double* g1,
               const double* l2, const Dims& d, cudaStream_t s) {
  k_e0<<<1, 1024, 0, s>>>(out, h, F, eri, g1, l2, d);
}
void launch_cumulant2(double* L2, double* D2, double* G, double* E, const double* g1,
                      const double* g2, int a, int given, cudaStream_t s) {
  if (a == 0) return;
  int64_t a4 = (int64_t)a * a * a * a;
  k_cumulant2<<<grid_for(a4), kThreads, 0, s>>>(L2, D2, G, E, g1, g2, a, given);
  k_direct2<<<grid_for(a4), kThreads, 0, s>>>(D2, L2, a);
}
void launch_direct3(double* D3, const double* L3, int a, cudaStream_t s) {
  if (a == 0) return;
  int64_t a6 = (int64_t)a * a * a * a * a * a;
  k_direct3<<<grid_for(a6), kThreads, 0, s>>>(D3, L3, a);
}

// ---------------------------------------------------------------------------
// Renormalised update (Eq. ric-update) and DIIS
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // v >= 0: the IEEE bit pattern orders like the value
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// T laid out as [T2 (np,np,nh,nh) | T1 (np,nh)]; R is X2 (needs the pair
// symmetrisation R = X + X^{pair}) followed by R1.
__global__ void k_update(const double* __restrict__ T, const double* __restrict__ X,
                         double* __restrict__ Tn, double* __restrict__ Err,
                         const double* __restrict__ eps, Dims d, double s, double* maxdt) {
  const int64_t np = d.np, nh = d.nh;
  const int64_t n2 = np * np * nh * nh, n1 = np * nh;
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2 + n1; i += (int64_t)gridDim.x * blockDim.x) {
    double t, r, D;
    bool zero;
    if (i < n2) {
      const int64_t c = i / (np * nh * nh), dd = (i / (nh * nh)) % np, k = (i / nh) % nh, l = i % nh;
      zero = (c < d.a && dd < d.a && k >= d.o && l >= d.o);
      t = T[i];
      r = X[i] + X[((dd * np + c) * nh + l) * nh + k];
      D = eps[k] + eps[l] - eps[d.o + c] - eps[d.o + dd];
    } else {
      const int64_t j = i - n2, c = j / nh, k = j % nh;
      zero = (c < d.a && k >= d.o);
      t = T[i];
      r = X[i];
      D = eps[k] - eps[d.o + c];
    }
    double tn = 0.0;
    if (!zero && D != 0.0) tn = (t * D + r) * (-expm1(-s * D * D) / D);
    Tn[i] = tn;
    const double e = tn - t;
    Err[i] = e;
    const double ae = fabs(e);
    mx = (ae > mx || ae != ae) ? ae : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double y = __shfl_down_sync(0xffffffffu, mx, o);
    mx = (y > mx || y != y) ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    if (mx != mx) mx = __longlong_as_double(0x7ff8000000000000LL);
    atomic_max_pos(maxdt, mx != mx ? 1.0e300 : mx);
  }
}

// dots[j] = sum_i E_new[i] * E_j[i] for j < m (history rows)
__global__ void k_dots(double* __restrict__ dots, const double* __restrict__ enew,
                       const double* __restrict__ hist, int64_t n, int m, int64_t ld) {
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      s = fma(enew[i], hist[j * ld + i], s);
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(dots + j, s);
  }
}

// Pulay system [B -1; -1 0] c = [0; -1] solved by Gaussian elimination with
// partial pivoting (m <= 16), single thread.  gram is m x m (ld 16).
__global__ void k_diis_solve(const double* __restrict__ gram, double* __restrict__ coef, int m,
                             int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double A[17][18];
  const int n = m + 1;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = gram[i * 16 + j];
    A[i][m] = -1.0;
    A[i][n] = 0.0;
  }
  for (int j = 0; j < m; ++j) A[m][j] = -1.0;
  A[m][m] = 0.0;
  A[m][n] = -1.0;
  int ok = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (!(fabs(A[piv][c]) > 1e-300)) { ok = 0; break; }
    if (piv != c)
      for (int j = 0; j <= n; ++j) { double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r][c] / A[c][c];
      for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
    }
  }
  if (ok) {
    double x[17];
    for (int r = n - 1; r >= 0; --r) {
      double s = A[r][n];
      for (int j = r + 1; j < n; ++j) s -= A[r][j] * x[j];
      x[r] = s / A[r][r];
    }
    for (int i = 0; i < m; ++i) {
      coef[i] = x[i];
      if (!(fabs(x[i]) < 1e300)) ok = 0;
    }
  }
  *status = ok;
}

// T = sum_j coef[j] * V_j  (falls back to the newest vector if status == 0)
__global__ void k_extrapolate(double* __restrict__ T, const double* __restrict__ vecs,
                              const double* __restrict__ coef, const int* status, int m,
                              int newest, int64_t n, int64_t ld) {
  const int ok = *status;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (ok) {
      for (int j = 0; j < m; ++j) s = fma(coef[j], vecs[j * ld + i], s);
    } else {
      s = vecs[newest * ld + i];
    }
    T[i] = s;
  }
}
}  // namespace

void launch_update(const double* T, const double* X, double* Tn, double* Err, const double* eps,
                   const Dims& d, double s, double* maxdt, cudaStream_t st) {
  int64_t n = (int64_t)d.np * d.np * d.nh * d.nh + (int64_t)d.np * d.nh;
  k_update<<<grid_for(n), kThreads, 0, st>>>(T, X, Tn, Err, eps, d, s, maxdt);
}
void launch_dots(double* dots, const double* enew, const double* hist, int64_t n, int m,
                 int64_t ld, cudaStream_t st) {
  k_dots<<<grid_for(n), kThreads, 0, st>>>(dots, enew, hist, n, m, ld);
}
void launch_diis_solve(const double* gram, double* coef, int m, int* status, cudaStream_t st) {
  k_diis_solve<<<1, 32, 0, st>>>(gram, coef, m, status);
}
void launch_extrapolate(double* T, const double* vecs, const double* coef, const int* status,
                        int m, int newest, int64_t n, int64_t ld, cudaStream_t st) {
  k_extrapolate<<<grid_for(n), kThreads, 0, st>>>(T, vecs, coef, status, m, newest, n, ld);
}

// ---------------------------------------------------------------------------
// Semi-canonicalisation: cyclic Jacobi on one symmetric block (one CTA)
// ---------------------------------------------------------------------------
namespace {
// *sweeps_done receives the sweeps performed, or -1 when max_sweeps sweeps
// left the off-diagonal norm above tol (not converged).
__global__ void k_jacobi(double* __restrict__ Ablk, double* __restrict__ V, int n, int max_sweeps,
                         double tol, int* sweeps_done) {
  // A (n x n, row-major) is overwritten; V accumulates rotations (V0 = I).
  __shared__ double cs[2];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  __shared__ double offs, tots;
  double tot = 0.0;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) tot += Ablk[i] * Ablk[i];
  tot = block_sum(tot);
  if (threadIdx.x == 0) tots = tot;
  __syncthreads();
  int sw = 0;
  for (;; ++sw) {
    double off = 0.0;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x)
      if (i / n != i % n) off += Ablk[i] * Ablk[i];
    off = block_sum(off);
    if (threadIdx.x == 0) offs = off;
    __syncthreads();
    if (offs <= tol * tol * tots) break;
    if (sw == max_sweeps) {
      sw = -1;
      break;
    }
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (threadIdx.x == 0) {
          const double apq = Ablk[p * n + q];
          double c = 1.0, s = 0.0;
          if (fabs(apq) > 1e-300) {
            const double app = Ablk[p * n + p], aqq = Ablk[q * n + q];
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          for (int k = threadIdx.x; k < n; k += blockDim.x) {  // columns p, q
            const double akp = Ablk[k * n + p], akq = Ablk[k * n + q];
            Ablk[k * n + p] = c * akp - s * akq;
            Ablk[k * n + q] = s * akp + c * akq;
          }
          __syncthreads();
          for (int k = threadIdx.x; k < n; k += blockDim.x) {  // rows p, q
            const double apk = Ablk[p * n + k], aqk = Ablk[q * n + k];
            Ablk[p * n + k] = c * apk - s * aqk;
            Ablk[q * n + k] = s * apk + c * aqk;
            const double vkp = V[k * n + p], vkq = V[k * n + q];
            V[k * n + p] = c * vkp - s * vkq;
            V[k * n + q] = s * vkp + c * vkq;
          }
        }
        __syncthreads();
      }
  }
  if (threadIdx.x == 0) *sweeps_done = sw;
}

// Sort eigenpairs ascending inside the block and fix signs (largest |v| > 0);
// write the block of U at (off, off) in the full n_full x n_full matrix.
__global__ void k_jacobi_finish(const double* __restrict__ Ablk, const double* __restrict__ V,
                                int n, double* __restrict__ U, int n_full, int off) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double w = Ablk[j * n + j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double wk = Ablk[k * n + k];
      if (wk < w || (wk == w && k < j)) ++rank;
    }
    int imax = 0;
    double vmax = -1.0;
    for (int k = 0; k < n; ++k)
      if (fabs(V[k * n + j]) > vmax) { vmax = fabs(V[k * n + j]); imax = k; }
    const double sg = V[imax * n + j] < 0 ? -1.0 : 1.0;
    for (int k = 0; k < n; ++k) U[(int64_t)(off + k) * n_full + off + rank] = sg * V[k * n + j];
  }
}
}  // namespace

// Convergence target of the off-diagonal norm relative to the Frobenius norm:
// 1e-15, loosened to n x 2.2e-16 for large blocks (the rounding floor of the
// rotations grows with n).  Returns the launches' own status.
cudaError_t run_jacobi(double* Ablk, double* V, int n, double* U, int n_full, int off, int* d_sweeps,
                       cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int max_sweeps = 40;
  double tol = n * 2.2e-16 > 1e-15 ? n * 2.2e-16 : 1e-15;
  void* a1[] = {&Ablk, &V, &n, &max_sweeps, &tol, &d_sweeps};
  cudaError_t e = cudaLaunchKernel((const void*)k_jacobi, dim3(1), dim3(1024), a1, 0, s);
  if (e != cudaSuccess) return e;
  void* a2[] = {(void*)&Ablk, (void*)&V, &n, &U, &n_full, &off};
  return cudaLaunchKernel((const void*)k_jacobi_finish, dim3(1), dim3(256), a2, 0, s);
}

namespace {
__global__ void k_energy_out(double* out, const double* acc, double e0) { *out = e0 + *acc; }
}  // namespace
void launch_energy_out(double* out, const double* acc, double e0, cudaStream_t s) {
  k_energy_out<<<1, 1, 0, s>>>(out, acc, e0);
}

// ---------------------------------------------------------------------------
// Adjoint of the renormalised fixed point (Lagrangian of G(T) = U(T) - T)
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ bool zero_block(int64_t i, const Dims& d, int64_t* c, int64_t* dd, int64_t* k,
                                           int64_t* l, bool* doubles) {
  const int64_t np = d.np, nh = d.nh, n2 = np * np * nh * nh;
  if (i < n2) {
    *doubles = true;
    *c = i / (np * nh * nh);
    *dd = (i / (nh * nh)) % np;
    *k = (i / nh) % nh;
    *l = i % nh;
    return *c < d.a && *dd < d.a && *k >= d.o && *l >= d.o;
  }
  *doubles = false;
  const int64_t j = i - n2;
  *c = j / nh;
  *k = j % nh;
  *dd = 0;
  *l = 0;
  return *c < d.a && *k >= d.o;
}
__device__ __forceinline__ double delta_of(const double* eps, const Dims& d, bool dbl, int64_t c, int64_t dd,
                                           int64_t k, int64_t l) {
  return dbl ? eps[k] + eps[l] - eps[d.o + c] - eps[d.o + dd] : eps[k] - eps[d.o + c];
}
__device__ __forceinline__ double phi_of(double D, double s) {
  return D == 0.0 ? 0.0 : -expm1(-s * D * D) / D;
}
// d phi / d Delta
__device__ __forceinline__ double dphi_of(double D, double s) {
  const double x = s * D * D;
  if (x < 1e-8) return s - 1.5 * s * s * D * D;
  return (2.0 * x * exp(-x) + expm1(-x)) / (D * D);
}

// Yraw = phi * Lam (zero outside the amplitude blocks); Ytil = Yraw with the
// doubles part pair-symmetrised, the weight of the raw doubles output X.
__global__ void k_adj_y(const double* __restrict__ Lam, double* __restrict__ Yraw, double* __restrict__ Ytil,
                        const double* __restrict__ eps, Dims d, double s) {
  const int64_t np = d.np, nh = d.nh, n2 = np * np * nh * nh, n = n2 + np * nh;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c, dd, k, l;
    bool dbl;
    const bool z = zero_block(i, d, &c, &dd, &k, &l, &dbl);
    Yraw[i] = z ? 0.0 : phi_of(delta_of(eps, d, dbl, c, dd, k, l), s) * Lam[i];
  }
}
__global__ void k_adj_sym(const double* __restrict__ Yraw, double* __restrict__ Ytil, Dims d) {
  const int64_t np = d.np, nh = d.nh, n2 = np * np * nh * nh, n = n2 + np * nh;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n2) {
      const int64_t c = i / (np * nh * nh), dd = (i / (nh * nh)) % np, k = (i / nh) % nh, l = i % nh;
      Ytil[i] = Yraw[i] + Yraw[((dd * np + c) * nh + l) * nh + k];
    } else {
      Ytil[i] = Yraw[i];
    }
  }
}
// Lam_new = S [Delta * Yraw + GT];  err = Lam_new - Lam;  max |err|.
// S averages each doubles element with its pair-swapped partner: the
// amplitudes live on the pair-symmetric subspace (Eq. spinfree-perm-sym), so
// the multipliers of the constrained fixed point are the projected ones.
__global__ void k_adj_update(const double* __restrict__ Lam, const double* __restrict__ Yraw,
                             const double* __restrict__ GT, double* __restrict__ Ln, double* __restrict__ Err,
                             const double* __restrict__ eps, Dims d, double* maxd) {
  const int64_t np = d.np, nh = d.nh, n2 = np * np * nh * nh, n = n2 + np * nh;
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c, dd, k, l;
    bool dbl;
    const bool z = zero_block(i, d, &c, &dd, &k, &l, &dbl);
    double v = 0.0;
    if (!z) {
      const double D = delta_of(eps, d, dbl, c, dd, k, l);  // pair-swap invariant
      v = D * Yraw[i] + GT[i];
      if (dbl) {
        const int64_t j = ((dd * np + c) * nh + l) * nh + k;
        v = 0.5 * (v + D * Yraw[j] + GT[j]);
      }
    }
    Ln[i] = v;
    const double e = v - Lam[i];
    Err[i] = e;
    const double ae = fabs(e);
    mx = (ae > mx || ae != ae) ? ae : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_down_sync(0xffffffffu, mx, o);
    mx = (y > mx || y != y) ? y : mx;
  }
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(maxd),
              (unsigned long long)__double_as_longlong(mx != mx ? 1.0e300 : mx));
}
// geps[p] += sum_nu Lam_nu dG_nu/dDelta_nu * dDelta_nu/deps_p and
// dEds += sum_nu Lam_nu (T Delta + R) dphi/ds, R = X + X^{pair}.
__global__ void k_adj_eps(const double* __restrict__ Lam, const double* __restrict__ T,
                          const double* __restrict__ X, const double* __restrict__ eps, Dims d, double s,
                          double* __restrict__ geps, double* __restrict__ dEds) {
  const int64_t np = d.np, nh = d.nh, n2 = np * np * nh * nh, n = n2 + np * nh;
  double acc_s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c, dd, k, l;
    bool dbl;
    if (zero_block(i, d, &c, &dd, &k, &l, &dbl)) continue;
    const double lam = Lam[i];
    if (lam == 0.0) continue;
    const double D = delta_of(eps, d, dbl, c, dd, k, l);
    const double r = dbl ? X[i] + X[((dd * np + c) * nh + l) * nh + k] : X[i];
    const double t = T[i];
    const double g = lam * (t * phi_of(D, s) + (t * D + r) * dphi_of(D, s));
    atomicAdd(geps + k, g);
    atomicAdd(geps + d.o + c, -g);
    if (dbl) {
      atomicAdd(geps + l, g);
      atomicAdd(geps + d.o + dd, -g);
    }
    acc_s += lam * (t * D + r) * D * exp(-s * D * D);
  }
  acc_s = block_sum(acc_s);
  if (threadIdx.x == 0) atomicAdd(dEds, acc_s);
}
// Chain through E0 = 1/2 sum D (h + f) + 1/2 sum (tu|vw) L2[t,v,u,w] and the
// Fock build f_pq = h_pq + sum_rs D_rs [(pq|rs) - 1/2 (ps|rq)]:
//   gFt = gF + diag(geps) + D/2 ;  gh = gFt + D/2
//   geri[p,q,r,s] += gFt[p,q] D[r,s] - 1/2 gFt[p,s] D[r,q] + 1/2 L2[p,r,q,s] (active)
// with D = 2 delta on the core, Gamma1 on the active block.
__device__ __forceinline__ double dens(const double* g1, const Dims& d, int64_t p, int64_t q) {
  if (p < d.o && q < d.o) return p == q ? 2.0 : 0.0;
  if (p >= d.o && q >= d.o && p < d.o + d.a && q < d.o + d.a) return g1[(p - d.o) * d.a + (q - d.o)];
  return 0.0;
}
__global__ void k_adj_fock(const double* __restrict__ gF, const double* __restrict__ geps,
                           const double* __restrict__ g1, Dims d, double* __restrict__ gFt, double* __restrict__ gh) {
  const int64_t n = d.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / n, q = i % n;
    const double D = dens(g1, d, p, q);
    const double v = gF[i] + (p == q ? geps[p] : 0.0) + 0.5 * D;
    gFt[i] = v;
    gh[i] = v + 0.5 * D;
  }
}
__global__ void k_adj_eri(double* __restrict__ geri, const double* __restrict__ gFt, const double* __restrict__ g1,
                          const double* __restrict__ l2, Dims d) {
  const int64_t n = d.n, nh = d.o + d.a, n2 = n * n, n3 = n2 * n, tot = n2 * n2;
  const int64_t a = d.a, a2 = a * a, a3 = a2 * a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / n3, q = (i / n2) % n, r = (i / n) % n, s = i % n;
    double v = 0.0;
    if (r < nh && s < nh) v += gFt[p * n + q] * dens(g1, d, r, s);
    if (r < nh && q < nh) v -= 0.5 * gFt[p * n + s] * dens(g1, d, r, q);
    if (a > 0 && p >= d.o && q >= d.o && r >= d.o && s >= d.o && p < nh && q < nh && r < nh && s < nh)
      v += 0.5 * l2[(p - d.o) * a3 + (r - d.o) * a2 + (q - d.o) * a + (s - d.o)];
    if (v != 0.0) geri[i] += v;
  }
}
// geri <- geri + geri^T over the (pq) <-> (rs) pair exchange (in place, upper triangle)
__global__ void k_sym_pairs(double* __restrict__ g, int64_t n2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2 * n2; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i / n2, y = i % n2;
    if (y < x) continue;
    const double a = g[x * n2 + y], b = g[y * n2 + x];
    g[x * n2 + y] = a + b;
    g[y * n2 + x] = a + b;
  }
}
}  // namespace

__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}
void launch_add(double* y, const double* x, int64_t n, cudaStream_t st) {
  k_add<<<grid_for(n), kThreads, 0, st>>>(y, x, n);
}
void launch_adj_y(const double* Lam, double* Yraw, double* Ytil, const double* eps, const Dims& d, double s,
                  cudaStream_t st) {
  const int64_t n = (int64_t)d.np * d.np * d.nh * d.nh + (int64_t)d.np * d.nh;
  k_adj_y<<<grid_for(n), kThreads, 0, st>>>(Lam, Yraw, Ytil, eps, d, s);
  k_adj_sym<<<grid_for(n), kThreads, 0, st>>>(Yraw, Ytil, d);
}
void launch_adj_update(const double* Lam, const double* Yraw, const double* GT, double* Ln, double* Err,
                       const double* eps, const Dims& d, double* maxd, cudaStream_t st) {
  const int64_t n = (int64_t)d.np * d.np * d.nh * d.nh + (int64_t)d.np * d.nh;
  k_adj_update<<<grid_for(n), kThreads, 0, st>>>(Lam, Yraw, GT, Ln, Err, eps, d, maxd);
}
void launch_adj_eps(const double* Lam, const double* T, const double* X, const double* eps, const Dims& d,
                    double s, double* geps, double* dEds, cudaStream_t st) {
  const int64_t n = (int64_t)d.np * d.np * d.nh * d.nh + (int64_t)d.np * d.nh;
  k_adj_eps<<<grid_for(n), kThreads, 0, st>>>(Lam, T, X, eps, d, s, geps, dEds);
}
void launch_adj_chain(double* geri, const double* gF, const double* geps, const double* g1, const double* l2,
                      const Dims& d, double* gFt, double* gh, cudaStream_t st) {
  const int64_t n = d.n;
  k_adj_fock<<<grid_for(n * n), kThreads, 0, st>>>(gF, geps, g1, d, gFt, gh);
  k_adj_eri<<<grid_for(n * n * n * n), kThreads, 0, st>>>(geri, gFt, g1, l2, d);
  k_sym_pairs<<<grid_for(n * n * n * n), kThreads, 0, st>>>(geri, n * n);
}
