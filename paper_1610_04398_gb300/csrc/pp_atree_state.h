// The device state pp_atree_solve keeps with an adaptive tree between calls (arrays of the tree
// and lists, expansions, the near-field table); released by pp_atree_destroy.
#pragma once

#include <vector>

#include "../../include/pp.h"

namespace pp {

// A tree and its lists in host memory, in the layout pp_atree_boxes / pp_atree_lists report;
// atree_adopt makes a pp_atree of it (the device build hands its results over this way).
struct AtreeHost {
    int max_level = 0;
    std::vector<int> level, ix, iy, parent, first_child, leaf;
    std::vector<int> m2l, p2p;
};
int atree_adopt(const AtreeHost& h, double theta, pp_atree* out);

void* atree_state(pp_atree t);
void atree_set_state(pp_atree t, void* state, void (*release)(void*));

}  // namespace pp
