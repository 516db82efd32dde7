"""The allocation-free index build caches the device address of its static
scratch per device and per CUDA context (the address belongs to the context
its module was loaded into).  Checked here on the CPU: the cache logic is a
template over its two lookups, compiled with fakes that count the lookups and
switch the current context."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_03174_b300", "csrc")

DRIVER = r'''
#include <stdio.h>
#include "noalloc_cache.h"
using namespace trd_host;
static unsigned long long g_ctx = 0;   // 0: no context current
static int g_lookups = 0;
static int32_t g_arena[4];
static bool ctx_id(unsigned long long *id) { if (!g_ctx) return false; *id = g_ctx; return true; }
static int lookup(int dev, NoAllocEntry *e) {
    ++g_lookups;
    if (!g_ctx) g_ctx = 100;                    // the lookup makes the primary context current
    e->scratch = g_arena + (g_ctx % 4);        // a new context may load the module elsewhere
    e->sm_count = 148 + dev;
    return 0;
}
static int fail_lookup(int, NoAllocEntry *) { ++g_lookups; return -4; }
#define CHECK(c) do { if (!(c)) { printf("FAIL line %d\n", __LINE__); return 1; } } while (0)
int main() {
    NoAllocEntry table[4] = {};
    std::mutex mu;
    NoAllocEntry e{};
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, lookup, &e) == 0);   // no context yet
    CHECK(g_lookups == 1 && e.scratch == g_arena + 0 && e.ctx_id == 100);
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, lookup, &e) == 0);   // cached
    CHECK(g_lookups == 1);
    g_ctx = 101;                                                        // context re-created
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, lookup, &e) == 0);
    CHECK(g_lookups == 2 && e.scratch == g_arena + 1 && e.ctx_id == 101);
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, lookup, &e) == 0);
    CHECK(g_lookups == 2);
    CHECK(noalloc_resolve(table, 4, mu, 1, ctx_id, lookup, &e) == 0);   // other device: own entry
    CHECK(g_lookups == 3 && e.sm_count == 149);
    g_ctx = 100;                                                        // back to an older id: looked up again
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, lookup, &e) == 0);
    CHECK(g_lookups == 4 && e.scratch == g_arena + 0);
    g_ctx = 102;
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, fail_lookup, &e) != 0);  // a failed lookup caches nothing
    CHECK(noalloc_resolve(table, 4, mu, 0, ctx_id, lookup, &e) == 0 && e.ctx_id == 102);
    CHECK(noalloc_resolve(table, 4, mu, 7, ctx_id, lookup, &e) != 0);   // device outside the table
    printf("ok\n");
    return 0;
}
'''


def test_noalloc_address_cache_is_dropped_when_the_context_changes(tmp_path):
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe), "-lpthread"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
