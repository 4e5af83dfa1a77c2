// Host build of the spectrum server's arena allocator (abcmb_arena.h).
#include "abcmb_arena.h"

static abcmb::Arena g_arena;

extern "C" void h_arena_init(size_t size) { g_arena.init(size); }
extern "C" int h_arena_alloc(size_t len, size_t *off) { return g_arena.alloc(len, off) ? 1 : 0; }
extern "C" void h_arena_release(size_t off, size_t len) { g_arena.release(off, len); }
extern "C" size_t h_arena_largest() { return g_arena.largest(); }
extern "C" size_t h_arena_size() { return g_arena.size(); }
