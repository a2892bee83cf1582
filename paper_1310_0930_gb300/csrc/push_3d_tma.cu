// push_3d_tma.cu -- instantiations of the particle kernel for the 3D entries of
// the tile menu (push_menu.h) that stage the field tile by TMA.
#define PIC_DIM 3
#define PIC_TMA true
#include "push_inst.h"

namespace pic {

cudaError_t launch_push_3d_tma(int order, const int *tile, int drift, const PushArgs &a, cudaStream_t st)
{
    PIC_PUSH_MENU_3D_TMA(PIC_PUSH_CASE)
    return cudaErrorInvalidValue;
}

size_t smem_push_3d_tma(int order, const int *tile, int drift)
{
    PIC_PUSH_MENU_3D_TMA(PIC_PUSH_SMEM)
    return 0;
}

int stage_push_3d_tma(int order, const int *tile, int drift, int *lo, int *len)
{
    PIC_PUSH_MENU_3D_TMA(PIC_PUSH_STAGE)
    return 0;
}

// extents of the TMA box of the field tile; 0 if not compiled
int box_push_3d_tma(int order, const int *tile, int drift, int *box)
{
    PIC_PUSH_MENU_3D_TMA(PIC_PUSH_BOX)
    return 0;
}

}  // namespace pic
