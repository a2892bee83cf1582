// push_q.cu -- the particle kernel at quartic order (the highest shape order
// of Table 3) for the default tile of each dimension: 3D 8x8x8 with drift 1,
// 2D 16x16 with drift 2.
#include "push.cuh"

namespace pic {

namespace {
template <class G>
int stage_q(int *lo, int *len)
{
    lo[0] = G::FHX;
    len[0] = G::FX;
    lo[1] = G::FHY;
    len[1] = G::FY;
    lo[2] = G::FHZ;
    len[2] = G::FZ;
    return 1;
}
using G3 = push_detail::Geo<3, 4, 8, 8, 8, 1, false>;
using G2 = push_detail::Geo<2, 4, 16, 16, 1, 2, false>;
bool is3(int dim, const int *tile, int drift)
{
    return dim == 3 && tile[0] == 8 && tile[1] == 8 && tile[2] == 8 && drift == 1;
}
bool is2(int dim, const int *tile, int drift) { return dim == 2 && tile[0] == 16 && tile[1] == 16 && drift == 2; }
}  // namespace

cudaError_t launch_push_q(int dim, const int *tile, int drift, const PushArgs &a, cudaStream_t st)
{
    if (is3(dim, tile, drift))
        return push_detail::launch_t<3, 4, 8, 8, 8, 1, false>(a.runs, a.items, a.nitems, a.block, a.tail_block, a.queue,
                                                             a.persistent_ctas, st, a.live_cnt, a.max_extra);
    if (is2(dim, tile, drift))
        return push_detail::launch_t<2, 4, 16, 16, 1, 2, false>(a.runs, a.items, a.nitems, a.block, a.tail_block,
                                                               a.queue, a.persistent_ctas, st, a.live_cnt,
                                                               a.max_extra);
    return cudaErrorInvalidValue;
}

size_t smem_push_q(int dim, const int *tile, int drift)
{
    if (is3(dim, tile, drift)) return G3::SMEM;
    if (is2(dim, tile, drift)) return G2::SMEM;
    return 0;
}

int stage_push_q(int dim, const int *tile, int drift, int *lo, int *len)
{
    if (is3(dim, tile, drift)) return stage_q<G3>(lo, len);
    if (is2(dim, tile, drift)) return stage_q<G2>(lo, len);
    return 0;
}

}  // namespace pic
