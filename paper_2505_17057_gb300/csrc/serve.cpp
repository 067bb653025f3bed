// serve.cpp -- solve server (filled in below the core solver).
#include "../../include/mmfd.h"

extern "C" {
int mmfd_server_create(const mmfd_server_desc*, mmfd_server**) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_submit(mmfd_server*, const mmfd_desc*, const void* const*, int, long long, unsigned long long*) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_poll(mmfd_server*, unsigned long long, mmfd_result*) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_server_drain(mmfd_server*) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_result_fields(mmfd_server*, unsigned long long, void* const*, int, int) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_release(mmfd_server*, unsigned long long) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_server_get_stats(const mmfd_server*, mmfd_server_stats*) { return MMFD_ERR_UNSUPPORTED; }
int mmfd_server_destroy(mmfd_server*) { return MMFD_OK; }
}
