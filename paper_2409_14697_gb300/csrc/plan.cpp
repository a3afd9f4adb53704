#include "plan.h"

namespace qs {

void run_planned(DeviceState &st, const std::vector<Op> &ops, const qs_options &o, qs_stats &stats) {
    (void)o;
    for (const Op &op : ops) {
        launch_stream_op(st, op);
        stats.passes++;
        stats.bytes += stream_bytes(op, st.n, st.dtype);
    }
    stats.ops_after_fuse = (int64_t)ops.size();
}

}  // namespace qs
