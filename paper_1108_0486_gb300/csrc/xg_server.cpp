// Request server (continuous batching); see xg_ctx::shutdown_server.
#include "xg_runtime.h"

void xg_ctx::shutdown_server() {}
