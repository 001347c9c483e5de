// Runs the library's double-float accumulation (dfloat.cuh) on the host:
//   dfloat_host N < taps (N floats) inputs (N doubles) > sum (2 doubles: s, c)
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1101_5803_gb300/csrc/dfloat.cuh"

int main(int argc, char** argv) {
    if (argc != 2) return 2;
    const int n = std::atoi(argv[1]);
    std::vector<float> t(n);
    std::vector<double> x(n);
    if (std::fread(t.data(), sizeof(float), n, stdin) != (size_t)n ||
        std::fread(x.data(), sizeof(double), n, stdin) != (size_t)n)
        return 2;
    float s = 0.f, c = 0.f;
    for (int i = 0; i < n; ++i) {
        float hi, lo;
        mirage::df_split(x[i], hi, lo);
        mirage::df_madd(s, c, t[i], hi, lo);
    }
    const double out[2] = {(double)s, (double)c};
    std::fwrite(out, sizeof(double), 2, stdout);
    return 0;
}
