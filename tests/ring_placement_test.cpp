// ring_placement_test.cpp -- the served kernel's tile placement in its CTA
// ring (push_lease in served_protocol.cuh, compiled for the host), checked
// on fixed cases.  Workers reserve ring positions in the order they become
// idle and write their warp next to the position; warp w runs on SM
// partition w % 4.  When the worker at a position runs on a partition that
// already holds a tile of the same lease, and a later waiting worker's
// partition is free, the agent queues an empty item there (the worker
// reserves again) so the lease's tiles spread over partitions.
//
// usage: ring_placement_test   (prints OK, or the first mismatch and exits 1)
#include "served_protocol.cuh"

#include <cstdio>
#include <vector>

using namespace srvp;

namespace {

int g_fail = 0;

struct Item {
    uint32_t t, nt;  // nt == 0: an empty item
};

// Workers with warps `warps` wait at positions tail .. tail + n - 1 (a warp
// of -1: reserved, owner word not written yet).
void wait_at(Ring &ring, uint32_t tail, const std::vector<int> &warps)
{
    ring.tail = tail;
    ring.head = tail + (uint32_t)warps.size();
    for (size_t i = 0; i < warps.size(); ++i) {
        const uint32_t pos = tail + (uint32_t)i;
        ring.owner[pos % kRing] = warps[i] < 0 ? ~0u : (pos << 8) | (uint32_t)warps[i];
    }
}

void expect(const char *name, Ring &ring, uint32_t tail, uint32_t pushed, uint32_t want_pushed,
            const std::vector<Item> &want, uint32_t used, uint32_t want_used)
{
    bool ok = pushed == want_pushed && ring.tail == tail + (uint32_t)want.size() && used == want_used;
    for (size_t i = 0; ok && i < want.size(); ++i) {
        const uint32_t s = (tail + (uint32_t)i) % kRing;
        ok = ring.t[s] == want[i].t && ring.nt[s] == want[i].nt && ring.d[s] == 7u && ring.seq[s] == 42u;
    }
    if (!ok) {
        ++g_fail;
        std::printf("FAIL %s: pushed %u (want %u), tail advanced by %u (want %zu), used %#x (want %#x); items:",
                    name, pushed, want_pushed, ring.tail - tail, want.size(), used, want_used);
        for (uint32_t i = 0; i < ring.tail - tail; ++i) {
            const uint32_t s = (tail + i) % kRing;
            std::printf(" (t %u, nt %u)", ring.t[s], ring.nt[s]);
        }
        std::printf("\n");
    }
}

void run_case(const char *name, uint32_t tail, const std::vector<int> &warps, uint32_t room, uint32_t lt,
              uint32_t lend, uint32_t used_in, uint32_t want_pushed, const std::vector<Item> &want,
              uint32_t want_used)
{
    Ring ring;
    ring_init(ring);
    wait_at(ring, tail, warps);
    uint32_t used = used_in;
    const uint32_t pushed = push_lease(ring, room, 7u, 42u, lt, lend, 100u, used);
    expect(name, ring, tail, pushed, want_pushed, want, used, want_used);
}

}  // namespace

int main()
{
    const uint32_t N = 100;  // the lease's request has 100 tiles
    // one worker per partition: the tiles go out in order
    run_case("distinct", 0, {1, 2, 3, 4}, 4, 0, 4, 0, 4, {{0, N}, {1, N}, {2, N}, {3, N}}, 0xf);
    // warps 1 and 5 share partition 1: the second gets an empty item, the
    // tile goes to the next free partition
    run_case("shared partition", 0, {1, 5, 2, 3, 4}, 5, 0, 4, 0, 4,
             {{0, N}, {1, 0}, {1, N}, {2, N}, {3, N}}, 0xf);
    // no later waiting worker on a free partition: no empty item
    run_case("no free partition later", 0, {1, 5}, 2, 0, 2, 0, 2, {{0, N}, {1, N}}, 0x2);
    // an owner word not written yet: placed as unknown, not marked used
    run_case("unknown owner", 0, {-1, 1, 5}, 3, 0, 3, 0, 3, {{0, N}, {1, N}, {2, N}}, 0x2);
    // room for fewer items than the lease has tiles: the rest stays
    run_case("room limits", 0, {1, 2}, 2, 0, 4, 0, 2, {{0, N}, {1, N}}, 0x6);
    // nobody waiting (queued ahead): tiles in order, no partition marked
    run_case("nobody waiting", 0, {}, 3, 5, 8, 0, 3, {{5, N}, {6, N}, {7, N}}, 0x0);
    // the lease continues: partitions used by its earlier tiles count (both
    // workers on partition 2 get empty items; tile 3 waits for more room)
    run_case("lease continues", 0, {2, 6, 3}, 3, 2, 4, 0x4, 1, {{2, 0}, {2, 0}, {2, N}}, 0xc);
    // positions wrap around the ring
    run_case("wrap", kRing - 2, {1, 5, 2}, 3, 0, 2, 0, 2, {{0, N}, {1, 0}, {1, N}}, 0x6);
    if (g_fail)
        return 1;
    std::printf("OK\n");
    return 0;
}
