// Host-side driver of the tuning cache (tune_lookup, tune_store, tune_key_rhs_block in
// csrc/lattices.cu), built and run by tests/test_tune_cache_cpu.py without a GPU.  The
// solver entry points that lattices.cu dispatches to are stubbed out: only the cache runs.
// Commands on standard input, one per line: "get <key>" prints the cached value or "none";
// "put <value> <key>" stores a value; "rhskey" prints a right-hand-side block key.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <iostream>
#include <string>

#include "../paper_1904_08616_gb300/csrc/lattices.cu"

namespace lq {
int fail(int status, const char*, ...) { return status; }
size_t spinor_bytes(int64_t, int) { return 0; }
size_t gauge_bytes(int64_t, int, int) { return 0; }
namespace solver_detail {
int lattices_f64(int, const LatticeJob*, const lq_cg_params&, double, char*, lq_cg_info*, cudaStream_t) { return 0; }
int lattices_f64x(int, const LatticeJob*, const lq_cg_params&, double, char*, lq_cg_info*, cudaStream_t) { return 0; }
int lattices_mixed_f32(int, const LatticeJob*, const lq_cg_params&, double, char*, lq_cg_info*, cudaStream_t) {
    return 0;
}
int lattices_mixed_f16(int, const LatticeJob*, const lq_cg_params&, double, char*, lq_cg_info*, cudaStream_t) {
    return 0;
}
}  // namespace solver_detail
}  // namespace lq

int main() {
    using namespace lq::solver_detail;
    std::string line;
    while (std::getline(std::cin, line)) {
        if (line.rfind("get ", 0) == 0) {
            int v = 0;
            if (tune_lookup(line.substr(4), &v)) printf("%d\n", v);
            else printf("none\n");
        } else if (line.rfind("put ", 0) == 0) {
            const size_t sp = line.find(' ', 4);
            tune_store(line.substr(sp + 1), atoi(line.substr(4, sp - 4).c_str()));
            printf("stored\n");
        } else if (line == "rhskey") {
            lq::Geom g{};
            g.L[0] = 8; g.L[1] = 6; g.L[2] = 4; g.L[3] = 6;
            printf("%s\n", tune_key_rhs_block(LQ_F16S, 12, LQ_F64X, g, 8).c_str());
        }
        fflush(stdout);
    }
    return 0;
}
