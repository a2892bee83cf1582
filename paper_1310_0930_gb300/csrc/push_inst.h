// push_inst.h -- dispatch of one file's share of the tile menu (push_menu.h)
// to the particle kernel instantiations of push.cuh.  A file defines
// PIC_DIM, PIC_TMA (field-tile layout) and PIC_MENU, then includes this.
#pragma once
#include "push.cuh"
#include "push_menu.h"

#define PIC_PUSH_CASE(TX, TY, TZ, D)                                                                         \
    if (tile[0] == TX && tile[1] == TY && (PIC_DIM == 2 || tile[2] == TZ) && drift == D) {                    \
        if (order == 1)                                                                                       \
            return push_detail::launch_t<PIC_DIM, 1, TX, TY, TZ, D, PIC_TMA>(                                 \
                a.runs, a.items, a.nitems, a.block, a.tail_block, a.queue, a.persistent_ctas, st, a.live_cnt, \
                a.max_extra);                                                                                 \
        if (order == 2)                                                                                       \
            return push_detail::launch_t<PIC_DIM, 2, TX, TY, TZ, D, PIC_TMA>(                                 \
                a.runs, a.items, a.nitems, a.block, a.tail_block, a.queue, a.persistent_ctas, st, a.live_cnt, \
                a.max_extra);                                                                                 \
        return push_detail::launch_t<PIC_DIM, 3, TX, TY, TZ, D, PIC_TMA>(                                     \
            a.runs, a.items, a.nitems, a.block, a.tail_block, a.queue, a.persistent_ctas, st, a.live_cnt,     \
            a.max_extra);                                                                                     \
    }
#define PIC_PUSH_SMEM(TX, TY, TZ, D)                                                                         \
    if (tile[0] == TX && tile[1] == TY && (PIC_DIM == 2 || tile[2] == TZ) && drift == D) {                    \
        if (order == 1) return push_detail::Geo<PIC_DIM, 1, TX, TY, TZ, D, PIC_TMA>::SMEM;                   \
        if (order == 2) return push_detail::Geo<PIC_DIM, 2, TX, TY, TZ, D, PIC_TMA>::SMEM;                   \
        return push_detail::Geo<PIC_DIM, 3, TX, TY, TZ, D, PIC_TMA>::SMEM;                                   \
    }
#define PIC_PUSH_STAGE(TX, TY, TZ, D)                                                                        \
    if (tile[0] == TX && tile[1] == TY && (PIC_DIM == 2 || tile[2] == TZ) && drift == D) {                    \
        if (order == 1) return stage_of<push_detail::Geo<PIC_DIM, 1, TX, TY, TZ, D, PIC_TMA>>(lo, len);      \
        if (order == 2) return stage_of<push_detail::Geo<PIC_DIM, 2, TX, TY, TZ, D, PIC_TMA>>(lo, len);      \
        return stage_of<push_detail::Geo<PIC_DIM, 3, TX, TY, TZ, D, PIC_TMA>>(lo, len);                      \
    }
#define PIC_PUSH_BOX(TX, TY, TZ, D)                                                                          \
    if (tile[0] == TX && tile[1] == TY && tile[2] == TZ && drift == D) {                                      \
        if (order == 1) return box_of<push_detail::Geo<3, 1, TX, TY, TZ, D, true>>(box);                     \
        if (order == 2) return box_of<push_detail::Geo<3, 2, TX, TY, TZ, D, true>>(box);                     \
        return box_of<push_detail::Geo<3, 3, TX, TY, TZ, D, true>>(box);                                     \
    }

namespace pic {
template <class G>
int stage_of(int *lo, int *len)
{
    lo[0] = G::FHX;
    len[0] = G::FX;
    lo[1] = G::FHY;
    len[1] = G::FY;
    lo[2] = G::FHZ;
    len[2] = G::FZ;
    return 1;
}
template <class G>
int box_of(int *box)
{
    box[0] = G::FX;
    box[1] = G::FY;
    box[2] = G::FZ;
    return 1;
}
}  // namespace pic
