// Temporary: entry points not built yet report ILU_EINVAL.
#include "../../include/ilu.h"
extern "C" {
ilu_status ilu_server_create(const ilu_server_opts *, ilu_server *) { return ILU_EINVAL; }
ilu_status ilu_server_submit(ilu_server, const ilu_request *, uint64_t *) { return ILU_EINVAL; }
ilu_status ilu_server_wait(ilu_server, uint64_t, int, ilu_result *) { return ILU_EINVAL; }
ilu_status ilu_server_release(ilu_server, uint64_t) { return ILU_EINVAL; }
ilu_status ilu_server_stats(ilu_server, ilu_stats *) { return ILU_EINVAL; }
ilu_status ilu_server_destroy(ilu_server) { return ILU_OK; }
}
