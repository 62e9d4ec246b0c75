// frame_r3.cu -- frame and batch kernels for a bilateral window of 7 x 7 quads (radius 3), one per
// Laplacian radius; split by bilateral radius so the three translation units compile in parallel.
#include "frame_kernels.cuh"

namespace pl3d {

const void* frame_kernel_rb3(int rl) {
    switch (rl) {
        case 1: return reinterpret_cast<const void*>(&frame_kernel<1, 3>);
        case 2: return reinterpret_cast<const void*>(&frame_kernel<2, 3>);
        case 3: return reinterpret_cast<const void*>(&frame_kernel<3, 3>);
        default: return nullptr;
    }
}

const void* batch_kernel_rb3(int rl) {
    switch (rl) {
        case 1: return reinterpret_cast<const void*>(&batch_kernel<1, 3>);
        case 2: return reinterpret_cast<const void*>(&batch_kernel<2, 3>);
        case 3: return reinterpret_cast<const void*>(&batch_kernel<3, 3>);
        default: return nullptr;
    }
}

}  // namespace pl3d
