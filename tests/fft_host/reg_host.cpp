// Runs the library's regulariser (reg.cuh) on the host:
//   reg_host SX SY REG < v (ns doubles) r (nreg doubles)
//   > H v (nreg doubles), H^T r (ns doubles), diag(H^T H) (ns doubles)
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1101_5803_gb300/csrc/reg.cuh"

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    mirage::Geo<double> g{};
    g.sx = std::atoi(argv[1]);
    g.sy = std::atoi(argv[2]);
    g.reg = std::atoi(argv[3]);
    g.ns = g.sx * g.sy;
    g.nreg = g.reg == 1 ? 2 * g.ns : g.ns;
    std::vector<double> v(g.ns), r(g.nreg), hv(g.nreg), htr(g.ns), d(g.ns);
    if ((int)std::fread(v.data(), 8, g.ns, stdin) != g.ns || (int)std::fread(r.data(), 8, g.nreg, stdin) != g.nreg)
        return 2;
    for (int row = 0; row < g.nreg; ++row) hv[row] = mirage::apply_H_row<double, double>(g, v.data(), row);
    for (int i = 0; i < g.ns; ++i) {
        const int ib = i / g.sx, ia = i - ib * g.sx;
        htr[i] = mirage::apply_HT_at<double, double>(g, r.data(), i, ia, ib);
        d[i] = mirage::hth_diag_at<double>(g, ia, ib);
    }
    std::fwrite(hv.data(), 8, hv.size(), stdout);
    std::fwrite(htr.data(), 8, htr.size(), stdout);
    std::fwrite(d.data(), 8, d.size(), stdout);
    return 0;
}
