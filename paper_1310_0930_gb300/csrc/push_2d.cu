// push_2d.cu -- instantiations of the particle kernel for the 2D entries of the
// tile menu (push_menu.h); the menu is split across files to compile in parallel.
#define PIC_DIM 2
#define PIC_TMA false
#include "push_inst.h"

namespace pic {

cudaError_t launch_push_2d(int order, const int *tile, int drift, const PushArgs &a, cudaStream_t st)
{
    PIC_PUSH_MENU_2D(PIC_PUSH_CASE)
    return cudaErrorInvalidValue;
}

size_t smem_push_2d(int order, const int *tile, int drift)
{
    PIC_PUSH_MENU_2D(PIC_PUSH_SMEM)
    return 0;
}

int stage_push_2d(int order, const int *tile, int drift, int *lo, int *len)
{
    PIC_PUSH_MENU_2D(PIC_PUSH_STAGE)
    return 0;
}

}  // namespace pic
