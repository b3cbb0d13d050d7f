// passes_f32.cu -- complex64 row/column pass launchers (N = 32 ... 8192).
#include "passes_launch.cuh"

namespace coro {

template <>
cudaError_t launch_row_pass<float2>(int n, const RowArgs<float2>& a, const PassLaunch& l) {
    using namespace detail;
    switch (n) {
        case 32: return row_launch<float2, 32>(a, l);
        case 64: return row_launch<float2, 64>(a, l);
        case 128: return row_launch<float2, 128>(a, l);
        case 256: return row_launch<float2, 256>(a, l);
        case 512: return row_launch<float2, 512>(a, l);
        case 1024: return row_launch_persistent<float2, 1024>(a, l);
        case 2048: return row_launch_persistent<float2, 2048>(a, l);
        case 4096: return row_launch_persistent<float2, 4096>(a, l);
        case 8192: return row_launch_persistent<float2, 8192>(a, l);
        default: return cudaErrorInvalidValue;
    }
}

// lines = columns per block; 0 = default. Wider blocks give longer contiguous segments per
// row (L * 8 bytes), narrower ones more resident blocks per SM.
template <>
cudaError_t launch_col_pass<float2>(int n, int lines, const ColArgs<float2>& a, const PassLaunch& l) {
    using namespace detail;
    if (lines == 0) lines = col_lines_default(n, false);
    switch (n) {
        case 32: return col_launch<float2, 32, 16>(a, l);
        case 64: return col_launch<float2, 64, 16>(a, l);
        case 128: return col_launch<float2, 128, 16>(a, l);
        case 256: return col_launch<float2, 256, 16>(a, l);
        case 512: return col_launch<float2, 512, 16>(a, l);
        case 1024: return lines == 8 ? col_launch<float2, 1024, 8>(a, l) : col_launch<float2, 1024, 16>(a, l);
        case 2048: return lines == 4 ? col_launch<float2, 2048, 4>(a, l) : col_launch<float2, 2048, 8>(a, l);
        case 4096: return lines == 2 ? col_launch<float2, 4096, 2>(a, l) : col_launch<float2, 4096, 4>(a, l);
        case 8192: return lines == 1 ? col_launch<float2, 8192, 1>(a, l) : col_launch<float2, 8192, 2>(a, l);
        default: return cudaErrorInvalidValue;
    }
}

int col_lines_default(int n, bool dbl) {
    if (dbl) {
        switch (n) {
            case 4096: return 1;
            case 2048: return 2;
            case 1024: return 4;
            case 512: case 256: return 8;
            default: return 16;
        }
    }
    switch (n) {
        case 8192: return 2;
        case 4096: return 4;
        case 2048: return 8;
        default: return 16;
    }
}

}  // namespace coro
