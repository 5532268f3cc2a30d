// Rule-specialised asynchronous kernel (host side).
//
// The general k_async interprets each rule's template (Sec. 2.2, ->int: the
// agents of Theta, their ports and the equations of Theta') from shared
// memory.  A rule set is fixed once loaded, so the same kernel can also be
// compiled with the templates as constants (k_async<kTrack, Rules>): a warp
// whose lanes all reduce one rule of at most two right-hand-side agents then
// runs that rule's straight-line code, with the values in registers.  This
// unit generates that source for a rule set, compiles it at run time with
// NVRTC (loaded with dlopen, so a missing NVRTC only turns the
// specialisation off), loads the cubin and keeps it for the process; cubins
// are also cached on disk, keyed by the templates, the embedded kernel
// sources, the NVRTC version and the architecture.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include "inet_layout.h"

namespace inet {

// Hash of the templates' bytes: the key a specialised kernel is built for.
// The host passes it in Dev::rules_key and the kernel refuses any other.
uint64_t rules_key(const Template* t, size_t n);

struct JitResult {
  const void* fn = nullptr;  // the kernel (a cudaKernel_t) for the runtime launch calls; null if not loaded
  double compile_ms = 0;     // NVRTC time (0 when the cubin came from a cache)
  bool from_disk = false;    // the cubin came from the on-disk cache
  bool from_memory = false;  // already loaded by this process
};

// The specialised k_async<track> for the n templates.  `load` false: compile
// (or find) the cubin only, without a device.  `arch`: "sm_103a" and the
// like.  Returns false with *err set when NVRTC is missing or fails.
bool jit_async(const Template* t, size_t n, bool track, const std::string& arch, bool load, JitResult* out,
               std::string* err);

// The generated source of the specialised kernel (for inspection and tests).
std::string jit_source(const Template* t, size_t n);

}  // namespace inet
