// passes_f64.cu -- complex128 row/column pass launchers (N = 32 ... 4096; other even N through
// the mixed-radix passes).
#include "passes_launch.cuh"
#include "mixed.cuh"

namespace coro {

template <>
cudaError_t launch_row_pass<double2>(int n, const RowArgs<double2>& a, const PassLaunch& l) {
    using namespace detail;
    switch (n) {
        case 32: return row_launch<double2, 32>(a, l);
        case 64: return row_launch<double2, 64>(a, l);
        case 128: return row_launch<double2, 128>(a, l);
        case 256: return row_launch<double2, 256>(a, l);
        case 512: return row_launch<double2, 512>(a, l);
        case 1024: return row_launch<double2, 1024>(a, l);
        case 2048: return row_launch<double2, 2048>(a, l);
        case 4096: return row_launch<double2, 4096>(a, l);
        default: return row_launch_mixed<double2>(n, a, l);
    }
}

template <>
cudaError_t launch_col_pass<double2>(int n, int lines, const ColArgs<double2>& a, const PassLaunch& l) {
    using namespace detail;
    (void)lines;
    switch (n) {
        case 32: return col_launch<double2, 32, 16>(a, l);
        case 64: return col_launch<double2, 64, 16>(a, l);
        case 128: return col_launch<double2, 128, 16>(a, l);
        case 256: return col_launch<double2, 256, 8>(a, l);
        case 512: return col_launch<double2, 512, 8>(a, l);
        case 1024: return col_launch<double2, 1024, 4>(a, l);
        case 2048: return col_launch<double2, 2048, 2>(a, l);
        case 4096: return col_launch<double2, 4096, 1>(a, l);
        default: return col_launch_mixed<double2>(n, 0, a, l);
    }
}

}  // namespace coro
