// frame_r2.cu -- frame and batch kernels for a bilateral window of 5 x 5 quads (radius 2), one per
// Laplacian radius; split by bilateral radius so the three translation units compile in parallel.
#include "frame_kernels.cuh"

namespace pl3d {

const void* frame_kernel_rb2(int rl) {
    switch (rl) {
        case 1: return reinterpret_cast<const void*>(&frame_kernel<1, 2>);
        case 2: return reinterpret_cast<const void*>(&frame_kernel<2, 2>);
        case 3: return reinterpret_cast<const void*>(&frame_kernel<3, 2>);
        default: return nullptr;
    }
}

const void* batch_kernel_rb2(int rl) {
    switch (rl) {
        case 1: return reinterpret_cast<const void*>(&batch_kernel<1, 2>);
        case 2: return reinterpret_cast<const void*>(&batch_kernel<2, 2>);
        case 3: return reinterpret_cast<const void*>(&batch_kernel<3, 2>);
        default: return nullptr;
    }
}

}  // namespace pl3d
