// Prints the library's bicubic weights (interp.cuh) for N offsets u in [0, 1]:
//   keys_host N > N x 4 doubles (weights of the centres at -1, 0, 1, 2)
#include <cstdio>
#include <cstdlib>

#include "../../paper_1101_5803_gb300/csrc/interp.cuh"

int main(int argc, char** argv) {
    if (argc != 2) return 2;
    const int n = std::atoi(argv[1]);
    for (int k = 0; k < n; ++k) {
        const double u = n > 1 ? (double)k / (n - 1) : 0.0;
        double w[4];
        for (int i = 0; i < 4; ++i) w[i] = mirage::keys_weight<double>(i, u);
        std::fwrite(w, sizeof(double), 4, stdout);
    }
    return 0;
}
