// The library's FFT convolution run by NT host threads as one CTA:
//   fft_host_mt NX NY K NT < image (NY*NX doubles) psf (K*K doubles) > B image, B^T image
// FP32 plan, as the inner solves use it; the spectrum is made by the same threads.
#include <barrier>
#include <cstdio>
#include <cstdlib>
#include <thread>
#include <vector>

#include "../../paper_1101_5803_gb300/csrc/fftconv.cuh"

thread_local HostDim threadIdx{0};
HostDim blockDim{1};
static std::barrier<>* g_bar = nullptr;
void host_cta_barrier() { g_bar->arrive_and_wait(); }

using namespace mirage;

int main(int argc, char** argv) {
    if (argc != 5) return 2;
    const int nx = std::atoi(argv[1]), ny = std::atoi(argv[2]), K = std::atoi(argv[3]), nt = std::atoi(argv[4]);
    std::vector<double> img((size_t)nx * ny), psf((size_t)K * K), outB((size_t)nx * ny), outT((size_t)nx * ny);
    if (std::fread(img.data(), 8, img.size(), stdin) != img.size() || std::fread(psf.data(), 8, psf.size(), stdin) != psf.size())
        return 2;
    const int M = std::max(16, fft_size_for(std::max(nx, ny) + (K - 1) / 2));
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    using C = float2;
    FftPlan<float> f;
    f.M = M;
    f.logM = logM;
    f.nb = fft_batch_count<C>(M);
    std::vector<C> tw(M - 1), buf((size_t)2 * f.nb * (M + 1)), F((size_t)(M / 2 + 1) * M), S((size_t)(M / 2 + 1) * M);
    std::vector<float> ps(psf.begin(), psf.end());
    f.tw = tw.data();
    f.b0 = buf.data();
    f.b1 = buf.data() + (size_t)f.nb * (M + 1);
    FftPlan<float> fs = f;
    fs.F = S.data();
    f.F = F.data();
    f.S = S.data();
    blockDim.x = (unsigned)nt;
    std::barrier<> bar(nt);
    g_bar = &bar;
    auto cta = [&](unsigned t) {
        threadIdx.x = t;
        fft_twiddles<float>(tw.data(), M);
        __syncthreads();
        fft_psf_spectrum<float>(fs, ps.data(), K);
        auto load = [&](int y, int n) -> float { return n < nx ? (float)img[(size_t)y * nx + n] : 0.f; };
        auto storeB = [&](int y, int n, float v) { outB[(size_t)y * nx + n] = v; };
        auto storeT = [&](int y, int n, float v) { outT[(size_t)y * nx + n] = v; };
        fft_convolve<float>(f, load, ny, storeB, ny, nx, false);
        fft_convolve<float>(f, load, ny, storeT, ny, nx, true);
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(cta, (unsigned)t);
    for (auto& x : th) x.join();
    std::fwrite(outB.data(), 8, outB.size(), stdout);
    std::fwrite(outT.data(), 8, outT.size(), stdout);
    return 0;
}
