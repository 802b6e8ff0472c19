// synth.cu -- pulse spectra and space-time synthesis by the discrete Fourier transform with the
// sign of Eq. (inverseFourier) (exp(-i omega t)), evaluated by a radix-2 FFT (Sec. 3 end:
// "discrete fast Fourier transform").
//   spectrum:  S[p][m] = sum_n s[p][n] exp(+2 pi i m n / Nt) = conj(FFT(s))_m  (real s)
//   synthesis: out[p][x][n] = (1/Nt) Re sum_m c_m exp(-2 pi i m n / Nt),  c_m = w_m S[p][m] T[m][x],
//              w_0 = w_{Nt/2} = 1, else 2 (the m > Nt/2 half is the complex conjugate).
// One CTA transforms one signal in shared memory with a Stockham (self-sorting) radix-2 FFT.
#include "bie_common.cuh"

namespace bie {

template <class S> struct C2 { S re, im; };

// tw[j] = exp(-2 pi i j / n), j < n/2, from sincospi (correctly rounded to ~1 ulp in FP64).
__global__ void k_twiddles(int n, double2* tw) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n / 2) return;
  double s, c;
  sincospi(2.0 * (double)j / (double)n, &s, &c);
  tw[j] = make_double2(c, -s);
}

// Forward FFT of buf (length n, power of two) in place, using tmp as the ping-pong partner.
// Returns the buffer that holds the result.
template <class S>
__device__ C2<S>* stockham(C2<S>* buf, C2<S>* tmp, int n, const double2* __restrict__ tw) {
  C2<S>* x = buf;
  C2<S>* y = tmp;
  for (int m = 1; m < n; m <<= 1) {
    const int twstep = n / (2 * m);
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int j = t / m, kk = t - j * m;
      const double2 w2 = tw[kk * twstep];
      const C2<S> w = {(S)w2.x, (S)w2.y};
      const C2<S> a = x[j * m + kk], b = x[j * m + kk + n / 2];
      const C2<S> wb = {w.re * b.re - w.im * b.im, w.re * b.im + w.im * b.re};
      y[2 * j * m + kk] = {a.re + wb.re, a.im + wb.im};
      y[2 * j * m + kk + m] = {a.re - wb.re, a.im - wb.im};
    }
    __syncthreads();
    C2<S>* t = x;
    x = y;
    y = t;
  }
  return x;
}

template <class S>
__global__ void k_pulse_spectrum(const double* __restrict__ s, int n, const double2* __restrict__ tw,
                                 cd* __restrict__ Sout) {
  extern __shared__ unsigned char smem_raw[];
  C2<S>* buf = reinterpret_cast<C2<S>*>(smem_raw);
  C2<S>* tmp = buf + n;
  const double* sp = s + (int64_t)blockIdx.x * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) buf[t] = {(S)sp[t], (S)0};
  __syncthreads();
  C2<S>* X = stockham<S>(buf, tmp, n, tw);
  cd* o = Sout + (int64_t)blockIdx.x * (n / 2 + 1);
  for (int t = threadIdx.x; t <= n / 2; t += blockDim.x) o[t] = {(double)X[t].re, -(double)X[t].im};
}

// grid: (M, P); one signal per CTA.
template <class S, class O>
__global__ void k_synth(const cd* __restrict__ T, const int64_t* __restrict__ midx, int nk, int64_t M,
                        const cd* __restrict__ Sp, int n, const double2* __restrict__ tw, O* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  C2<S>* buf = reinterpret_cast<C2<S>*>(smem_raw);
  C2<S>* tmp = buf + n;
  const int64_t x = blockIdx.x;
  const int p = blockIdx.y;
  for (int t = threadIdx.x; t < n; t += blockDim.x) buf[t] = {(S)0, (S)0};
  __syncthreads();
  const cd* Srow = Sp + (int64_t)p * (n / 2 + 1);
  for (int r = threadIdx.x; r < nk; r += blockDim.x) {
    const int m = (int)midx[r];
    const double w = (m == 0 || 2 * m == n) ? 1.0 : 2.0;
    const cd a = cmul(Srow[m], T[(int64_t)r * M + x]);
    buf[m] = {(S)(w * a.re), (S)(w * a.im)};
  }
  __syncthreads();
  C2<S>* X = stockham<S>(buf, tmp, n, tw);
  O* o = out + ((int64_t)p * M + x) * n;
  const S inv = (S)1 / (S)n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) o[t] = (O)(X[t].re * inv);
}

static int twiddle_table(bie_ctx* c, int n, double2** tw) {
  BIE_TRY(ensure_buf(c->work2, (size_t)(n / 2 + 1) * sizeof(double2)));
  *tw = (double2*)c->work2.p;
  k_twiddles<<<(n / 2 + 255) / 256, 256, 0, c->stream>>>(n, *tw);
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int pulse_spectrum(bie_ctx* c, const double* s, int64_t P, int n, cd* Sout) {
  double2* tw;
  BIE_TRY(twiddle_table(c, n, &tw));
  size_t smem = 2 * (size_t)n * sizeof(C2<double>);
  BIE_CUDA_TRY(cudaFuncSetAttribute(k_pulse_spectrum<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_pulse_spectrum<double><<<(unsigned)P, std::min(512, n / 2), smem, c->stream>>>(s, n, tw, Sout);
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int synthesize(bie_ctx* c, const cd* T, const int64_t* midx_dev, int nk, int64_t M, const cd* Sp, int64_t P, int n,
               void* out, int out_dtype) {
  double2* tw;
  BIE_TRY(twiddle_table(c, n, &tw));
  dim3 g((unsigned)M, (unsigned)P);
  int threads = std::min(512, std::max(32, n / 2));
  if (out_dtype == 0) {
    size_t smem = 2 * (size_t)n * sizeof(C2<double>);
    BIE_CUDA_TRY(cudaFuncSetAttribute(k_synth<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_synth<double, double><<<g, threads, smem, c->stream>>>(T, midx_dev, nk, M, Sp, n, tw, (double*)out);
  } else {
    size_t smem = 2 * (size_t)n * sizeof(C2<float>);
    BIE_CUDA_TRY(cudaFuncSetAttribute(k_synth<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_synth<float, float><<<g, threads, smem, c->stream>>>(T, midx_dev, nk, M, Sp, n, tw, (float*)out);
  }
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
