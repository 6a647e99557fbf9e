// serve.cu -- placeholder until the continuous-batching server lands.
#include "server.h"

namespace prnu {
struct Server::Impl {};
Server::Server(prnu_ctx*) {}
Server::~Server() {}
int Server::submit(const prnu_query*, uint64_t*) { set_error("serving not built"); return PRNU_EINVAL; }
int Server::poll(uint64_t, prnu_result*, int64_t) { set_error("serving not built"); return PRNU_EINVAL; }
void Server::stats(prnu_server_stats* out) { *out = prnu_server_stats{}; }
}  // namespace prnu

extern "C" {
int query_submit(prnu_ctx*, const prnu_query*, uint64_t*) { prnu::set_error("serving not built"); return PRNU_EINVAL; }
int query_poll(prnu_ctx*, uint64_t, prnu_result*, int64_t) { prnu::set_error("serving not built"); return PRNU_EINVAL; }
int prnu_server_stats_get(prnu_ctx*, prnu_server_stats* out) { if (out) *out = prnu_server_stats{}; return PRNU_OK; }
}
