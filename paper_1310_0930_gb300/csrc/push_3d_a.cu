// push_3d_a.cu -- instantiations of the particle kernel for 3D entries of the
// tile menu (push_menu.h), plain field-tile staging.
#define PIC_DIM 3
#define PIC_TMA false
#include "push_inst.h"

namespace pic {

cudaError_t launch_push_3d_a(int order, const int *tile, int drift, const PushArgs &a, cudaStream_t st)
{
    PIC_PUSH_MENU_3D_A(PIC_PUSH_CASE)
    return cudaErrorInvalidValue;
}

size_t smem_push_3d_a(int order, const int *tile, int drift)
{
    PIC_PUSH_MENU_3D_A(PIC_PUSH_SMEM)
    return 0;
}

int stage_push_3d_a(int order, const int *tile, int drift, int *lo, int *len)
{
    PIC_PUSH_MENU_3D_A(PIC_PUSH_STAGE)
    return 0;
}

}  // namespace pic
