// Runs the library's lens model (lens.cuh) on the host:
//   lens_host < N_LENS, per lens: 7 doubles, N_RAYS, 2*N_RAYS doubles (x, y)
//   > per lens: bad (int32), then 2*N_RAYS doubles (beta_x, beta_y)
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../paper_1101_5803_gb300/csrc/lens.cuh"

int main() {
    int32_t nl = 0;
    if (std::fread(&nl, 4, 1, stdin) != 1) return 2;
    for (int k = 0; k < nl; ++k) {
        double p[7];
        int32_t nr = 0;
        if (std::fread(p, 8, 7, stdin) != 7 || std::fread(&nr, 4, 1, stdin) != 1 || nr < 0) return 2;
        std::vector<double> xy(2 * (size_t)nr), out(2 * (size_t)nr);
        if (std::fread(xy.data(), 8, xy.size(), stdin) != xy.size()) return 2;
        const mirage::LensT<double> L = mirage::make_lens<double>(p);
        for (int i = 0; i < nr; ++i) mirage::trace_ray(L, xy[2 * i], xy[2 * i + 1], out[2 * i], out[2 * i + 1]);
        const int32_t bad = L.bad;
        std::fwrite(&bad, 4, 1, stdout);
        std::fwrite(out.data(), 8, out.size(), stdout);
    }
    return 0;
}
