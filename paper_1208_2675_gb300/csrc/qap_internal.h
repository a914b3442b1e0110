// qap_internal.h -- library-internal hooks shared by the translation units of
// libqapsa (not part of the C ABI; hidden symbols).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "qap_sa.h"

// The stream a handle issues its work on.
cudaStream_t qapsa_handle_stream(qap_sa *h);
// SMs one chain of size N occupies while it runs (1, or its cluster size).
int qapsa_sms_for(int N);
// Device bytes a chain of size N holds while it runs (set-up peak included).
size_t qapsa_bytes_for(int N);
// Keeps a cluster-tier handle in Delta mode for its whole run (a no-op for
// the one-SM tier): its run is then one launch per piece, which holds the
// cluster's SMs throughout.  Used by the server, where a second launch after a
// Delta rebuild waited for a free cluster of SMs while still counted as
// running.  The trajectory is the same in every mode.
void qapsa_keep_delta_mode(qap_sa *h);
