// Build-time generator: writes the hierarchic basis tables of basis.cpp as
// __device__ constexpr arrays, so that the operator kernels see every table
// entry as a compile-time constant (structurally zero entries then cost
// nothing).  Usage: gen_tables <output.inc>
#include <cmath>
#include <cstdio>

#include "rve_internal.h"

int main(int argc, char** argv) {
    if (argc < 2) return 2;
    FILE* f = std::fopen(argv[1], "w");
    if (!f) return 1;
    std::fprintf(f, "// Generated at build time by gen_tables.cpp from basis.cpp; not edited by hand.\n");
    std::fprintf(f, "// A[k][m][j]: coefficient of d phi_j / d xi_k on the orthonormal mode m of P_{p-1}.\n");
    std::fprintf(f, "namespace ctab {\n");
    for (int p = 1; p <= 3; ++p) {
        const rve::Basis& B = rve::basis(p);
        for (int fl = 0; fl < 2; ++fl) {
            std::fprintf(f, "__device__ constexpr %s A%d%s[%zu] = {", fl ? "float" : "double", p, fl ? "f" : "",
                         B.A.size());
            for (size_t i = 0; i < B.A.size(); ++i) {
                const double v = (std::fabs(B.A[i]) < 1e-14) ? 0.0 : B.A[i];
                if (fl)
                    std::fprintf(f, "%s%.9ef", i ? ", " : "", (double)(float)v);
                else
                    std::fprintf(f, "%s%.17e", i ? ", " : "", v);
            }
            std::fprintf(f, "};\n");
        }
    }
    std::fprintf(f, "}  // namespace ctab\n");
    std::fclose(f);
    return 0;
}
