// Amplitude server: placeholder until the request loop lands.
#include "plan.h"

extern "C" {
int tz_server_create(const tz_server_opts *, tz_server **out) {
  if (out) *out = nullptr;
  return TZ_EUNSUPPORTED;
}
int tz_server_submit(tz_server *, tz_plan *, const uint8_t *, int64_t, uint64_t *) { return TZ_EUNSUPPORTED; }
int tz_server_poll(tz_server *, uint64_t, double *, int *) { return TZ_EUNSUPPORTED; }
int tz_server_latency(tz_server *, double *, double *, int64_t *) { return TZ_EUNSUPPORTED; }
void tz_server_destroy(tz_server *) {}
}
