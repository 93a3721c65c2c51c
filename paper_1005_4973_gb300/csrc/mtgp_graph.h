// The constructor behind mtgp_graph_create, shared by the host library and the
// server (host code only; not part of the public C ABI).
#pragma once

#include "mtgp.h"

namespace mtgp {

// allow_pieces = false: the captured launch never splits a work item into
// jump-ahead pieces (Sec. 7), whatever the pool's configuration.
mtgp_status graph_create(mtgp_pool *p, uint32_t max_items, void *stream, bool allow_pieces, mtgp_graph **out);

}  // namespace mtgp
