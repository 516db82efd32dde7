// noalloc_cache.h -- the device address of the allocation-free entry point's
// static scratch, cached per device and per CUDA context.
//
// In host code the scratch array's name is only a host-side stand-in; its
// device address comes from cudaGetSymbolAddress, with the device current.
// That address belongs to the context the module was loaded into: after the
// primary context is torn down and created again (cudaDeviceReset, say) the
// module is loaded again and the array may sit elsewhere.  So an entry is
// used only while the current context is the one it was looked up in; any
// other context makes the next call look the address up again.  The logic is
// a template over its two lookups so that it can be checked on a machine
// without a GPU.
#pragma once

#include <stdint.h>

#include <mutex>

namespace trd_host {

struct NoAllocEntry {
    unsigned long long ctx_id;  // context the address was looked up in
    int32_t *scratch;           // device address of the scratch array there
    int sm_count;
    bool valid;
};

// ctx_id(&id) -> bool: the current context's id, false when none is current.
// lookup(dev, &entry) -> int: 0 and the entry's scratch and sm_count filled
// in, with dev current; a negative error code otherwise.
template <class CtxId, class Lookup>
int noalloc_resolve(NoAllocEntry *table, int n_dev, std::mutex &mu, int dev, CtxId ctx_id, Lookup lookup,
                    NoAllocEntry *out)
{
    if (dev < 0 || dev >= n_dev) return -4;
    unsigned long long id = 0;
    const bool have = ctx_id(&id);
    std::lock_guard<std::mutex> g(mu);
    NoAllocEntry &e = table[dev];
    if (have && e.valid && e.ctx_id == id) {
        *out = e;
        return 0;
    }
    NoAllocEntry fresh{};
    const int rc = lookup(dev, &fresh);  // makes the device's context current if none was
    if (rc) return rc;
    if (!ctx_id(&id)) return -4;
    fresh.ctx_id = id;
    fresh.valid = true;
    e = fresh;
    *out = fresh;
    return 0;
}

}  // namespace trd_host
