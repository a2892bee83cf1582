// push_split.cu -- the particle kernel with the virtual-trajectory deposit
// (Sec. 5.2 step iv) for the default tile of each dimension (3D 8x8x8 with
// drift 1, 2D 16x16 with drift 2), orders 1 to 3.
#include "push.cuh"

namespace pic {

namespace {
template <class G>
int stage_s(int *lo, int *len)
{
    lo[0] = G::FHX;
    len[0] = G::FX;
    lo[1] = G::FHY;
    len[1] = G::FY;
    lo[2] = G::FHZ;
    len[2] = G::FZ;
    return 1;
}
constexpr int kS = push_detail::kVarSplit;
template <int P>
using G3 = push_detail::Geo<3, P, 8, 8, 8, 1, kS>;
template <int P>
using G2 = push_detail::Geo<2, P, 16, 16, 1, 2, kS>;
bool is3(int dim, const int *tile, int drift)
{
    return dim == 3 && tile[0] == 8 && tile[1] == 8 && tile[2] == 8 && drift == 1;
}
bool is2(int dim, const int *tile, int drift) { return dim == 2 && tile[0] == 16 && tile[1] == 16 && drift == 2; }

template <int DIM, int P>
cudaError_t launch_s(const PushArgs &a, cudaStream_t st)
{
    if (DIM == 3)
        return push_detail::launch_t<3, P, 8, 8, 8, 1, kS>(a.runs, a.items, a.nitems, a.block, a.tail_block, a.queue,
                                                          a.persistent_ctas, st, a.live_cnt, a.max_extra);
    return push_detail::launch_t<2, P, 16, 16, 1, 2, kS>(a.runs, a.items, a.nitems, a.block, a.tail_block, a.queue,
                                                        a.persistent_ctas, st, a.live_cnt, a.max_extra);
}
}  // namespace

cudaError_t launch_push_split(int dim, int order, const int *tile, int drift, const PushArgs &a, cudaStream_t st)
{
    if (is3(dim, tile, drift)) {
        if (order == 1) return launch_s<3, 1>(a, st);
        if (order == 2) return launch_s<3, 2>(a, st);
        if (order == 3) return launch_s<3, 3>(a, st);
    }
    if (is2(dim, tile, drift)) {
        if (order == 1) return launch_s<2, 1>(a, st);
        if (order == 2) return launch_s<2, 2>(a, st);
        if (order == 3) return launch_s<2, 3>(a, st);
    }
    return cudaErrorInvalidValue;
}

size_t smem_push_split(int dim, int order, const int *tile, int drift)
{
    if (is3(dim, tile, drift)) {
        if (order == 1) return G3<1>::SMEM;
        if (order == 2) return G3<2>::SMEM;
        if (order == 3) return G3<3>::SMEM;
    }
    if (is2(dim, tile, drift)) {
        if (order == 1) return G2<1>::SMEM;
        if (order == 2) return G2<2>::SMEM;
        if (order == 3) return G2<3>::SMEM;
    }
    return 0;
}

int stage_push_split(int dim, int order, const int *tile, int drift, int *lo, int *len)
{
    if (is3(dim, tile, drift)) {
        if (order == 1) return stage_s<G3<1>>(lo, len);
        if (order == 2) return stage_s<G3<2>>(lo, len);
        if (order == 3) return stage_s<G3<3>>(lo, len);
    }
    if (is2(dim, tile, drift)) {
        if (order == 1) return stage_s<G2<1>>(lo, len);
        if (order == 2) return stage_s<G2<2>>(lo, len);
        if (order == 3) return stage_s<G2<3>>(lo, len);
    }
    return 0;
}

}  // namespace pic
