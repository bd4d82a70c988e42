"""The measurement protocol of bench.py, checked on the CPU: which workloads
must flush L2 between timed steps (a database that fits on chip would be
read from L2 after the first query), the algorithmic bytes the rooflines
divide by, and that ncu-measured DRAM traffic is only reported for the grid
it was captured on."""
import bench


def test_l2_flush_only_for_databases_that_fit_on_chip():
    small = bench.WORKLOADS["exact_packed_1k_64"]
    big = bench.WORKLOADS["exact_packed_50k_128"]
    assert bench.algorithmic_bytes(small) < 2 * bench.L2_BYTES
    assert bench.algorithmic_bytes(big) > 100 * bench.L2_BYTES
    assert bench.FLUSH_BYTES > bench.L2_BYTES


def test_algorithmic_bytes_of_the_packed_scan():
    # 50,000 x 128^3: two planes of 65,536 words plus two mask sizes per
    # entry, and the patient's two planes once
    wl = bench.WORKLOADS["exact_packed_50k_128"]
    plane = (128 ** 3 // 32) * 4
    assert bench.algorithmic_bytes(wl) == wl["n"] * (2 * plane + 8) + 2 * plane == 26_215_324_288


def test_traffic_reported_only_for_the_captured_grid():
    t = bench.TRAFFIC["scan_packed_kernel"]
    full = bench._traffic("scan_packed_kernel", 50_000, (128, 128, 128))
    assert bench._traffic("scan_packed_kernel", 1_024, (64, 64, 64)) is None
    assert bench._traffic("no_such_kernel", 10, (128, 128, 128)) is None
    if full is not None:      # None once the kernel's sources change
        assert abs(full - (t["read_bytes"] / t["entries"] * 50_000 + t["write_bytes"])) < 1.0


def test_support_words_match_the_support_lists_definition():
    """The sparse loops read every 16-byte word of each 64-byte granule of a
    plane where the patient's mask is non-zero (fewer words in a final
    partial granule): the bench's byte count, against a direct count."""
    import numpy as np
    import torch
    rng = np.random.default_rng(0)
    for shape in ((128, 128, 128), (30, 17, 11), (64, 64, 64), (9, 10, 11)):
        nx, ny, nz = shape
        vol = np.zeros((nz, ny, nx), np.float32)
        z0 = int(rng.integers(0, nz // 2 + 1))
        dz = min(max(1, nz // 4), nz - z0)
        vol[z0:z0 + dz, : max(1, ny // 3), :] = rng.random((dz, max(1, ny // 3), nx),
                                                            dtype=np.float32)
        got = bench._support_granules(torch, torch.from_numpy(vol), 0.6, 0.25)
        v = nx * ny * nz
        wp4 = ((v + 31) // 32 + 3) // 4
        want = 0
        for t in (np.float32(0.6), np.float32(0.25)):
            m = np.zeros(wp4 * 128, bool)
            m[:v] = vol.reshape(-1) >= t
            word_nz = m.reshape(wp4, 128).any(axis=1)
            for g in range((wp4 + 3) // 4):
                if word_nz[4 * g:4 * g + 4].any():
                    want += min(4, wp4 - 4 * g)
        assert got == want, (shape, got, want)
