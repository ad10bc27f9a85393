"""The benchmark's per-kernel algorithmic byte counts (the numerators of
its roofline fractions) follow the per-unit figures documented for each
kernel; checked on the 1M-Gaussian frame's sizes."""
import bench

N, M, T = 1_000_000, 11_765_641, 3600


def test_frame_kernels():
    ab = bench.algorithmic_bytes
    assert ab("frame_count", N, N, M, T) == 28 * N
    assert ab("preprocess_count", N, N, M, T) == 92 * N
    assert ab("preprocess", N, N, M, T) == 80 * N
    # single-launch depth sort: three 16-byte passes plus the depth-order scan
    assert ab("depth_sort", N, N, M, T, depth_passes=-3) == 16 * N * 3 + 12 * N
    # one launch per pass
    assert ab("depth_sort", N, N, M, T, depth_passes=1) == 16 * N
    # the count step and the depth sort in one launch: record in, 3 passes, offsets
    assert ab("count_depth_sort", N, N, M, T, depth_passes=-3) == 16 * N + 16 * N * 3 + 8 * N
    assert ab("duplicate_by_depth", N, N, M, T) == 32 * N + 4 * M
    assert ab("tile_sort_pass", M, N, M, T) == 8 * M
    assert ab("tile_expand_pass", M, N, M, T) == 16 * M + 8 * N + 16 * T == 196_307_856


def test_separate_steps():
    ab = bench.algorithmic_bytes
    assert ab("count_tiles", N, N, M, T) == 20 * N
    assert ab("scan", N, N, M, T) == 8 * N
    assert ab("duplicate_keys", N, N, M, T) == 20 * N + 12 * M
    assert ab("radix_pass", M, N, M, T) == 24 * M
    assert ab("tile_ranges", M, N, M, T) == 8 * M + 8 * T
    assert ab("unknown_kernel", M, N, M, T) == 0.0


def test_host_cpu_description():
    s = bench.host_cpu()
    assert "logical cores" in s
