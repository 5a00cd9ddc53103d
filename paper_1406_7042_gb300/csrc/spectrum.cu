// Frequency-domain post-processing of probe waveforms: discrete Fourier
// transform at chosen frequencies, resonance extraction and S-parameters (the
// spectra from which the paper reads its resonance frequencies, Sec. V-A, and
// S11, S21, Sec. V-D).  Y_p(f) = sum_n w_n y^n_p exp(-j 2 pi f t_n) dt with
// t_n = (n + 1) dt (y^n samples E^{n+1}) and the optional Hann window
// w_n = sin^2(pi (n + 1/2) / N).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"

namespace fdtdmor {

// One CTA per (frequency, probe): FP64 sums over the samples.
template <typename T>
__global__ void __launch_bounds__(256) dft_kernel(const T *__restrict__ y, int64_t nsteps, int p, double dt,
                                                  const double *__restrict__ freqs, int hann, double *__restrict__ out) {
  __shared__ double sr[256 / 32], si[256 / 32];
  const int fi = blockIdx.x, pi = blockIdx.y;
  const double f = freqs[fi];
  double re = 0.0, im = 0.0;
  for (int64_t n = threadIdx.x; n < nsteps; n += blockDim.x) {
    double w = 1.0;
    if (hann) {
      const double sw = sinpi((n + 0.5) / (double)nsteps);
      w = sw * sw;
    }
    // exp(-j 2 pi f t_n): the argument in units of pi, reduced modulo 2
    const double arg = fmod(2.0 * f * (double)(n + 1) * dt, 2.0);
    double s, c;
    sincospi(arg, &s, &c);
    const double v = w * (double)y[n * p + pi];
    re += v * c;
    im -= v * s;
  }
  for (int o = 16; o; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sr[w]; b += si[w]; }
    out[((size_t)pi * gridDim.x + fi) * 2] = a * dt;
    out[((size_t)pi * gridDim.x + fi) * 2 + 1] = b * dt;
  }
}

static fdtd_status dft_host(const void *y, int64_t nsteps, int p, fdtd_prec prec, double dt, int nf,
                            const double *freqs, int hann, double *out, cudaStream_t s) {
  DevBuf df, dout;
  struct Rel {
    DevBuf *a, *b;
    cudaStream_t s;
    ~Rel() { a->release(s); b->release(s); }
  } rel{&df, &dout, s};
  FDTD_CHECK(df.alloc(sizeof(double) * nf, s));
  FDTD_CHECK(dout.alloc(sizeof(double) * 2 * (size_t)nf * p, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(df.ptr, freqs, sizeof(double) * nf, cudaMemcpyHostToDevice, s));
  const dim3 grid(nf, p);
  if (prec == FDTD_F64)
    dft_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(y), nsteps, p, dt, df.as<double>(), hann,
                                            dout.as<double>());
  else
    dft_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(y), nsteps, p, dt, df.as<double>(), hann,
                                           dout.as<double>());
  FDTD_CHECK(after_launch("dft_kernel"));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(out, dout.ptr, sizeof(double) * 2 * (size_t)nf * p, cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status fdtd_dft(const void *y, int64_t nsteps, int p, fdtd_prec prec, double dt, int nf, const double *freqs,
                     int hann, double *out, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(y && freqs && out, "fdtd_dft: NULL argument");
  FDTD_REQUIRE(nsteps >= 1 && p >= 1 && p <= 65535 && nf >= 1 && dt > 0, "fdtd_dft: bad sizes");
  FDTD_REQUIRE(prec == FDTD_F32 || prec == FDTD_F64, "fdtd_dft: prec must be FDTD_F32 or FDTD_F64");
  return dft_host(y, nsteps, p, prec, dt, nf, freqs, hann, out, (cudaStream_t)stream);
}

fdtd_status fdtd_sparams(const void *y, const void *y_inc, int64_t nsteps, int p, fdtd_prec prec, double dt, int nf,
                         const double *freqs, int hann, int port_in, double *out, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(y && y_inc && freqs && out, "fdtd_sparams: NULL argument");
  FDTD_REQUIRE(p >= 1 && port_in >= 0 && port_in < p, "fdtd_sparams: port_in must be in [0, p)");
  FDTD_REQUIRE(nf >= 1, "fdtd_sparams: nf must be >= 1");
  std::vector<double> Y(2 * (size_t)nf * p), Yi(2 * (size_t)nf * p);
  FDTD_CHECK(fdtd_dft(y, nsteps, p, prec, dt, nf, freqs, hann, Y.data(), stream));
  FDTD_CHECK(fdtd_dft(y_inc, nsteps, p, prec, dt, nf, freqs, hann, Yi.data(), stream));
  for (int i = 0; i < nf; ++i) {
    const size_t ii = ((size_t)port_in * nf + i) * 2;
    const std::complex<double> inc(Yi[ii], Yi[ii + 1]);
    FDTD_REQUIRE(std::abs(inc) > 0, "fdtd_sparams: the incident spectrum vanishes at frequency %d", i);
    for (int q = 0; q < p; ++q) {
      const size_t k = ((size_t)q * nf + i) * 2;
      std::complex<double> num(Y[k], Y[k + 1]);
      if (q == port_in) num -= inc;
      const std::complex<double> sq = num / inc;
      out[k] = sq.real();
      out[k + 1] = sq.imag();
    }
  }
  return FDTD_OK;
}

fdtd_status fdtd_resonances(const void *y, int64_t nsteps, int p, fdtd_prec prec, double dt, double fmin,
                            double fmax, int nf, int hann, double rel_floor, int npk, double *peaks_hz, int *nfound,
                            fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(peaks_hz && nfound && npk >= 1, "fdtd_resonances: NULL output or npk < 1");
  FDTD_REQUIRE(nf >= 3 && fmax > fmin && fmin >= 0, "fdtd_resonances: need nf >= 3 and 0 <= fmin < fmax");
  std::vector<double> f(nf), Y(2 * (size_t)nf * p);
  for (int i = 0; i < nf; ++i) f[i] = fmin + (fmax - fmin) * i / (nf - 1);
  FDTD_CHECK(fdtd_dft(y, nsteps, p, prec, dt, nf, f.data(), hann, Y.data(), stream));
  // summed magnitude over the probes
  std::vector<double> mag(nf, 0.0);
  for (int q = 0; q < p; ++q)
    for (int i = 0; i < nf; ++i) mag[i] += std::hypot(Y[((size_t)q * nf + i) * 2], Y[((size_t)q * nf + i) * 2 + 1]);
  const double top = *std::max_element(mag.begin(), mag.end());
  std::vector<std::pair<double, double>> pk;  // (magnitude, refined frequency)
  for (int i = 1; i + 1 < nf; ++i) {
    if (!(mag[i] > mag[i - 1] && mag[i] >= mag[i + 1] && mag[i] >= rel_floor * top)) continue;
    // vertex of the parabola through the three samples
    const double a = mag[i - 1], b = mag[i], c = mag[i + 1];
    const double den = a - 2 * b + c;
    const double off = den != 0 ? 0.5 * (a - c) / den : 0.0;
    pk.push_back({b, f[i] + off * (f[1] - f[0])});
  }
  std::sort(pk.begin(), pk.end(), [](const auto &x, const auto &z) { return x.first > z.first; });
  const int n = std::min<int>(npk, (int)pk.size());
  std::vector<double> fr;
  for (int i = 0; i < n; ++i) fr.push_back(pk[i].second);
  std::sort(fr.begin(), fr.end());
  for (int i = 0; i < n; ++i) peaks_hz[i] = fr[i];
  *nfound = n;
  return FDTD_OK;
}

}  // extern "C"
