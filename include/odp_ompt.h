/*
 * odp_ompt.h -- the OMPT front end, libodp_ompt.so.
 *
 * An OpenMP runtime with the OMPT tools interface (OpenMP 5.1: target,
 * target-data-op and target-submit callbacks in their EMI form) loads the
 * library through OMP_TOOL_LIBRARIES=<path>/libodp_ompt.so and calls its
 * ompt_start_tool.  The tool then records every device allocation, delete,
 * transfer and kernel launch as an odp_event (times from the begin and end
 * callbacks, the host for the runtime's initial device, code locations
 * numbered by return address), fingerprints each transfer on the GPU when
 * its bytes are in device memory, and submits the events to an odp_server
 * on device 0, which streams the paper's findings (Sec. 5, Alg. 1-5) while
 * the program runs.  At the runtime's finalize it flushes the server, runs
 * odp_analyze over the log and prints the counts to stderr; with
 * ODP_OMPT_OUT=<prefix> it writes <prefix>.events (the log, 64-byte
 * records) and <prefix>.sites ("id address" per line).  ODP_OMPT_DISABLE=1
 * makes ompt_start_tool decline; ODP_OMPT_MAX_EVENTS sets the log capacity
 * (default 2^22), and with it the device memory the server reserves
 * (odp_server_bytes).  If the server cannot be created the tool prints why
 * and stays inactive (its initializer returns 0).
 *
 * The paper's tool hashes on the host CPU during the transfer; this one
 * hashes on the GPU, synchronously, so a kernel cannot change the bytes
 * first.  Asynchronous data operations are fingerprinted at their end
 * callback, which assumes the runtime issues it after the copy completed.
 */
#ifndef ODP_OMPT_H
#define ODP_OMPT_H

#include <stdint.h>

#include "odp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The tool's server (null before the runtime initialised the tool, or if
 * it could not start); its findings can be polled with odp_server_poll. */
odp_server* odp_ompt_server(void);

/* Events the tool could not record (fingerprint or submit failures). */
uint64_t odp_ompt_dropped(void);

/* Destroys the tool's server (after the runtime's finalize). */
void odp_ompt_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* ODP_OMPT_H */
