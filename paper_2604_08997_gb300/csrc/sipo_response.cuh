// Material response front and back end (Sec. 2.1; Eqs. 4-5, 28, 46): the
// generalised logistic (Richards) response m = M(f) of a resin to dose f, its
// inverse, and the response-domain post-scaling and metrics of a solved dose.
#pragma once

#include <math_constants.h>

#include "sipo_device.cuh"

namespace sipo {

// M(f) = alpha + (k - alpha) / [1 + exp(-beta (f - f0))]^(1/gamma)   (Eq. 4)
struct Richards {
  double alpha, k, beta, gamma, f0;
};

__device__ __forceinline__ double richards(const Richards& r, double f) {
  return r.alpha + (r.k - r.alpha) / pow(1.0 + exp(-r.beta * (f - r.f0)), 1.0 / r.gamma);
}

// M^-1(m) = f0 - ln[((k - alpha) / (m - alpha))^gamma - 1] / beta   (Eq. 5),
// defined for alpha < m < k.
__device__ __forceinline__ double richards_inverse(const Richards& r, double m) {
  return r.f0 - log(pow((r.k - r.alpha) / (m - r.alpha), r.gamma) - 1.0) / r.beta;
}

// Elementwise map of v = scale * in.  inverse = 0: out = M(v).  inverse = 1:
// out = M^-1(v) for alpha < v < k, 0 for v <= alpha (no prescription: outside
// the part); a value >= k (outside the invertible range) or NaN is counted in
// *n_bad and written as 0.
__global__ void k_response_map(const float* in, float* out, long long n, Richards r, double scale,
                               int inverse, unsigned long long* n_bad) {
  unsigned long long bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = scale * double(in[i]);
    double o;
    if (!inverse) {
      o = richards(r, v);
    } else if (v <= r.alpha) {
      o = 0.0;
    } else if (v < r.k) {
      o = richards_inverse(r, v);
    } else {
      ++bad;
      o = 0.0;
    }
    out[i] = float(o);
  }
  if (bad) atomicAdd(n_bad, bad);
}

// Phi_m(alpha_j) = sum_gel (M(alpha_j d_i) - m_T,i)^2 for K candidate factors
// (Eq. 28 with unit weights): per block and candidate, part[j * gridDim.x + b].
constexpr int kPhiCand = 32;

template <typename C>
__global__ void __launch_bounds__(kThreads) k_response_phi(const C* __restrict__ d, const uint8_t* __restrict__ lab,
                                                           const float* __restrict__ mT, Richards r,
                                                           const double* __restrict__ alphas, long long n,
                                                           double* __restrict__ part) {
  __shared__ double a_s[kPhiCand];
  if (threadIdx.x < kPhiCand) a_s[threadIdx.x] = alphas[threadIdx.x];
  __syncthreads();
  double acc[kPhiCand];
#pragma unroll
  for (int j = 0; j < kPhiCand; ++j) acc[j] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (lab[i] != kGel) continue;
    const double di = double(d[i]), mi = double(mT[i]);
#pragma unroll 4
    for (int j = 0; j < kPhiCand; ++j) {
      const double e = richards(r, a_s[j] * di) - mi;
      acc[j] += e * e;
    }
  }
  __shared__ double sh[kThreads];
  for (int j = 0; j < kPhiCand; ++j) {
    sh[threadIdx.x] = acc[j];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// At one factor alpha: min and max over gel of M(alpha d_i) / m_T,i, max over
// band of M(alpha d_i), min over gel of M(alpha d_i); per block, slot-major.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_response_ratio(const C* __restrict__ d, const uint8_t* __restrict__ lab,
                                                             const float* __restrict__ mT, Richards r,
                                                             double alpha, long long n,
                                                             double* __restrict__ part) {
  double v[4] = {1e300, -1e300, -1e300, 1e300};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t l = lab[i];
    if (l == kExt) continue;
    const double m = richards(r, alpha * double(d[i]));
    if (l == kBand) {
      v[2] = fmax(v[2], m);
    } else {
      const double q = m / double(mT[i]);
      v[0] = fmin(v[0], q);
      v[1] = fmax(v[1], q);
      v[3] = fmin(v[3], m);
    }
  }
  __shared__ double sh[kThreads];
  for (int j = 0; j < 4; ++j) {
    sh[threadIdx.x] = v[j];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        const double a = sh[threadIdx.x], b = sh[threadIdx.x + st];
        sh[threadIdx.x] = (j == 0 || j == 3) ? fmin(a, b) : fmax(a, b);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// Case 2 with a response threshold (Sec. 2.7.2 through Eq. 5): the smallest
// prescribed response over the part (values above the lower asymptote alpha),
// as ordered bits of a float, then the ratio M^-1(m_crit) / M^-1(min m_T).
__device__ __forceinline__ unsigned int ordered_bits(float x) {
  const unsigned int b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_response_gel_min(const float* __restrict__ mT, long long n, double alpha,
                                   unsigned int* __restrict__ out) {
  unsigned int best = 0xffffffffu;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float m = mT[i];
    if (double(m) > alpha) best = min(best, ordered_bits(m));  // NaN fails the test
  }
  atomicMin(out, best);
}

// One thread: ratio = M^-1(m_crit) / M^-1(gel minimum), NaN when either is
// outside (alpha, k) or no response lies above alpha.
__global__ void k_response_case2_ratio(const unsigned int* __restrict__ mn, Richards r, double m_crit,
                                       double* __restrict__ ratio, double* __restrict__ gel_min) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double g = *mn == 0xffffffffu ? CUDART_NAN : double(from_ordered_bits(*mn));
  *gel_min = g;
  const bool ok = g > r.alpha && g < r.k && m_crit > r.alpha && m_crit < r.k;
  *ratio = ok ? richards_inverse(r, m_crit) / richards_inverse(r, g) : CUDART_NAN;
}

}  // namespace sipo
