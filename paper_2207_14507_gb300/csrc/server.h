// server.h -- continuous-batching query server of a prnu context.
#pragma once
#include "internal.h"

namespace prnu {

class Server {
 public:
  explicit Server(prnu_ctx* ctx);
  ~Server();
  int submit(const prnu_query* q, uint64_t* qid);
  int poll(uint64_t qid, prnu_result* out, int64_t timeout_us);
  void stats(prnu_server_stats* out);
  bool latency(uint64_t qid, double* queued_ms, double* total_ms);

 private:
  struct Impl;
  std::unique_ptr<Impl> impl_;
};

}  // namespace prnu
