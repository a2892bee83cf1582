// push.cu -- dispatch of the particle kernel over the compiled tile menu.
#include "internal.h"

namespace pic {

cudaError_t launch_push_2d(int, const int *, int, const Run *, const Item *, int, int, int, int *, int, cudaStream_t);
cudaError_t launch_push_3d_a(int, const int *, int, const Run *, const Item *, int, int, int, int *, int, cudaStream_t);
cudaError_t launch_push_3d_b(int, const int *, int, const Run *, const Item *, int, int, int, int *, int, cudaStream_t);
cudaError_t launch_push_3d_tma(int, const int *, int, const Run *, const Item *, int, int, int, int *, int,
                               cudaStream_t);
size_t smem_push_2d(int, const int *, int);
size_t smem_push_3d_a(int, const int *, int);
size_t smem_push_3d_b(int, const int *, int);
size_t smem_push_3d_tma(int, const int *, int);
int box_push_3d_tma(int, const int *, int, int *);

int push_default_drift(int dim, const int *tile)
{
    if (dim == 3) return 1;
    if (tile[0] == 16) return 2;
    if (tile[0] == 8) return 1;
    return 2;
}

size_t push_smem_bytes(int dim, int order, const int *tile, int drift, bool tma)
{
    if (dim == 2) return tma ? 0 : smem_push_2d(order, tile, drift);
    if (tma) return smem_push_3d_tma(order, tile, drift);
    size_t s = smem_push_3d_a(order, tile, drift);
    return s ? s : smem_push_3d_b(order, tile, drift);
}

int push_tma_box(int dim, int order, const int *tile, int drift, int *box)
{
    return dim == 3 ? box_push_3d_tma(order, tile, drift, box) : 0;
}

cudaError_t launch_push(int dim, int order, const int *tile, int drift, bool tma, const Run *runs, const Item *items,
                        int nitems, int block, int tail_block, int *queue, int persistent_ctas, cudaStream_t st)
{
    if (dim == 2)
        return launch_push_2d(order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas, st);
    if (tma)
        return launch_push_3d_tma(order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas,
                                  st);
    if (smem_push_3d_a(order, tile, drift))
        return launch_push_3d_a(order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas, st);
    return launch_push_3d_b(order, tile, drift, runs, items, nitems, block, tail_block, queue, persistent_ctas, st);
}

}  // namespace pic
