// serve.cu -- the serving loop (continuous batching).
#include "host.h"

namespace hjcd {

struct Server {};

void server_stop(hjcd_ctx* ctx) {
    delete ctx->server;
    ctx->server = nullptr;
}

}  // namespace hjcd
