// push.cu -- dispatch of the particle kernel over the compiled tile menu.
#include "internal.h"

namespace pic {

cudaError_t launch_push_2d(int, int, const int *, int, const Run *, const Item *, int, int, int, int *, int, cudaStream_t);
cudaError_t launch_push_3d_a(int, int, const int *, int, const Run *, const Item *, int, int, int, int *, int, cudaStream_t);
cudaError_t launch_push_3d_b(int, int, const int *, int, const Run *, const Item *, int, int, int, int *, int, cudaStream_t);
size_t push_smem_2d(int, int, const int *, int);
size_t push_smem_3d_a(int, int, const int *, int);
size_t push_smem_3d_b(int, int, const int *, int);

int push_default_drift(int dim, const int *tile)
{
    if (dim == 3) return 1;
    if (tile[0] == 16) return 2;
    if (tile[0] == 8) return 1;
    return 2;
}

size_t push_smem_bytes(int dim, int order, const int *tile, int drift)
{
    if (dim == 2) return push_smem_2d(dim, order, tile, drift);
    size_t s = push_smem_3d_a(dim, order, tile, drift);
    return s ? s : push_smem_3d_b(dim, order, tile, drift);
}

cudaError_t launch_push(int dim, int order, const int *tile, int drift, const Run *runs, const Item *items,
                        int nitems, int block, int tail_block, int *queue, int persistent_ctas, cudaStream_t st)
{
    if (dim == 2)
        return launch_push_2d(dim, order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas, st);
    if (push_smem_3d_a(dim, order, tile, drift))
        return launch_push_3d_a(dim, order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas,
                                st);
    return launch_push_3d_b(dim, order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas,
                            st);
}

}  // namespace pic
