// Runs the library's L-curve corner (lcurve.cuh) on the host for many curves:
//   lcurve_host < N_CURVES, then per curve: n, chi2[n], reg[n] (int32 + doubles)
//   > per curve: corner (int32), flat (int32), kappa[n] (doubles)
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../paper_1101_5803_gb300/csrc/lcurve.cuh"

int main() {
    int32_t nc = 0;
    if (std::fread(&nc, 4, 1, stdin) != 1) return 2;
    for (int c = 0; c < nc; ++c) {
        int32_t n = 0;
        if (std::fread(&n, 4, 1, stdin) != 1 || n < 0 || n > mirage::MAX_LAM) return 2;
        std::vector<double> chi2(n), reg(n), kappa(mirage::MAX_LAM, 0.0);
        if ((int)std::fread(chi2.data(), 8, n, stdin) != n || (int)std::fread(reg.data(), 8, n, stdin) != n) return 2;
        int flat = 0;
        const int32_t corner = mirage::lcurve_corner_dev(chi2.data(), reg.data(), n, kappa.data(), &flat);
        const int32_t fl = flat;
        std::fwrite(&corner, 4, 1, stdout);
        std::fwrite(&fl, 4, 1, stdout);
        std::fwrite(kappa.data(), 8, n, stdout);
    }
    return 0;
}
