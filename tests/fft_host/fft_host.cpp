// Runs the library's FFT convolution (fftconv.cuh) on the host for one image:
//   fft_host NX NY K PREC CORR < image (NY*NX doubles) psf (K*K doubles)
//   > output (NY*NX doubles)
// PREC 32 or 64; CORR 1 for B^T.  Grid side as the library picks it:
// the smallest power of two >= max(NX, NY) + (K-1)/2, at least 16.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1101_5803_gb300/csrc/fftconv.cuh"

using namespace mirage;

template <typename R>
static int run(int nx, int ny, int K, bool corr, const std::vector<double>& img, const std::vector<double>& psf,
               std::vector<double>& out) {
    using C = typename CxOf<R>::type;
    int M = std::max(16, fft_size_for(std::max(nx, ny) + (K - 1) / 2));
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    FftPlan<R> f;
    f.M = M;
    f.logM = logM;
    f.nb = fft_batch_count<C>(M);
    std::vector<C> tw(M - 1), buf((size_t)2 * f.nb * (M + 1)), F((size_t)(M / 2 + 1) * M), S((size_t)(M / 2 + 1) * M);
    std::vector<R> ps(psf.begin(), psf.end());
    fft_twiddles<R>(tw.data(), M);
    f.tw = tw.data();
    f.b0 = buf.data();
    f.b1 = buf.data() + (size_t)f.nb * (M + 1);
    FftPlan<R> fs = f;
    fs.F = S.data();
    fft_psf_spectrum<R>(fs, ps.data(), K);
    f.F = F.data();
    f.S = S.data();
    auto load = [&](int y, int n) -> R { return n < nx ? (R)img[(size_t)y * nx + n] : (R)0; };
    auto store = [&](int y, int n, R v) { out[(size_t)y * nx + n] = (double)v; };
    fft_convolve<R>(f, load, ny, store, ny, nx, corr);
    return M;
}

int main(int argc, char** argv) {
    if (argc != 6) {
        std::fprintf(stderr, "usage: fft_host NX NY K PREC CORR\n");
        return 2;
    }
    const int nx = std::atoi(argv[1]), ny = std::atoi(argv[2]), K = std::atoi(argv[3]);
    const int prec = std::atoi(argv[4]);
    const bool corr = std::atoi(argv[5]) != 0;
    std::vector<double> img((size_t)nx * ny), psf((size_t)K * K), out((size_t)nx * ny, 0.0);
    if (std::fread(img.data(), sizeof(double), img.size(), stdin) != img.size() ||
        std::fread(psf.data(), sizeof(double), psf.size(), stdin) != psf.size()) {
        std::fprintf(stderr, "short input\n");
        return 2;
    }
    const int M = prec == 32 ? run<float>(nx, ny, K, corr, img, psf, out) : run<double>(nx, ny, K, corr, img, psf, out);
    std::fwrite(out.data(), sizeof(double), out.size(), stdout);
    std::fprintf(stderr, "M=%d\n", M);
    return 0;
}
