// Chunk planner + in-cache executor (Sec. II-B "Qubit Reordering", "In-cache Operations";
// Sec. III-A tiers 4-5; Sec. III-B).
#pragma once
#include "qs_internal.h"

namespace qs {

// Plans `ops` into passes and launches them on st.stream, filling stats.
void run_planned(DeviceState &st, const std::vector<Op> &ops, const qs_options &o, qs_stats &stats);

}  // namespace qs
