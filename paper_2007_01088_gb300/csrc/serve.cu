// Serving loop (placeholder).
#include "cc3_internal.h"

extern "C" {
int cc3_serve_start(cc3_server **out, size_t, int) { if (out) *out = nullptr; return CC3_ERR_UNSUPPORTED; }
int cc3_serve_submit(cc3_server *, const cc3_request *, uint64_t *) { return CC3_ERR_UNSUPPORTED; }
int cc3_serve_poll(cc3_server *, uint64_t, int *) { return CC3_ERR_UNSUPPORTED; }
int cc3_serve_wait(cc3_server *, uint64_t, double) { return CC3_ERR_UNSUPPORTED; }
int cc3_serve_cancel(cc3_server *, uint64_t) { return CC3_ERR_UNSUPPORTED; }
int cc3_serve_stats(cc3_server *, cc3_stats *) { return CC3_ERR_UNSUPPORTED; }
int cc3_serve_stop(cc3_server *) { return CC3_ERR_UNSUPPORTED; }
}
