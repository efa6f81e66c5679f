// The device state pp_atree_solve keeps with an adaptive tree between calls (arrays of the tree
// and lists, expansions, the near-field table); released by pp_atree_destroy.
#pragma once

#include "../../include/pp.h"

namespace pp {

void* atree_state(pp_atree t);
void atree_set_state(pp_atree t, void* state, void (*release)(void*));

}  // namespace pp
