// Error-message hooks that the host mesh structure (mesh_accel.cpp) expects from the rest of
// libetac, so that file can be built alone with the address and undefined-behaviour
// sanitizers for tests/test_sanitizers.py.  Test infrastructure only.
#include <string>

static thread_local std::string g_err;

namespace etac {
void set_context_free_error(const std::string& msg) { g_err = msg; }
}  // namespace etac

extern "C" const char* etac_last_error(const void*) { return g_err.c_str(); }
