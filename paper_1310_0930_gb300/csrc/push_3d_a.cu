// push_3d_a.cu -- instantiations of the particle kernel (push.cuh) for the
// 3D entries of push_menu.h; split across files to compile in parallel.
#include "push.cuh"
#include "push_menu.h"

namespace pic {

#define PIC_PUSH_CASE(TX, TY, TZ, D)                                                                \
    if (tile[0] == TX && tile[1] == TY && (dim == 2 || tile[2] == TZ) && drift == D) {               \
        if (order == 1) return push_detail::launch_t<3, 1, TX, TY, TZ, D>(runs, items, nitems, block, tail_block, queue, persistent_ctas, st); \
        if (order == 2) return push_detail::launch_t<3, 2, TX, TY, TZ, D>(runs, items, nitems, block, tail_block, queue, persistent_ctas, st); \
        return push_detail::launch_t<3, 3, TX, TY, TZ, D>(runs, items, nitems, block, tail_block, queue, persistent_ctas, st);             \
    }
#define PIC_PUSH_SMEM(TX, TY, TZ, D)                                                                 \
    if (tile[0] == TX && tile[1] == TY && (dim == 2 || tile[2] == TZ) && drift == D) {               \
        if (order == 1) return push_detail::Geo<3, 1, TX, TY, TZ, D>::SMEM;                    \
        if (order == 2) return push_detail::Geo<3, 2, TX, TY, TZ, D>::SMEM;                    \
        return push_detail::Geo<3, 3, TX, TY, TZ, D>::SMEM;                                    \
    }

cudaError_t launch_push_3d_a(int dim, int order, const int *tile, int drift, const Run *runs, const Item *items,
                           int nitems, int block, int tail_block, int *queue, int persistent_ctas, cudaStream_t st)
{
    PIC_PUSH_MENU_3D_A(PIC_PUSH_CASE)
    return cudaErrorInvalidValue;
}

size_t push_smem_3d_a(int dim, int order, const int *tile, int drift)
{
    PIC_PUSH_MENU_3D_A(PIC_PUSH_SMEM)
    return 0;
}

}  // namespace pic
