"""Host-side measurement arithmetic of bench.py (no GPU): the algorithmic bytes per launch that
the roofline divides by the measured launch time, counted array by array at mMR scale, and the
whole-job rate of the replicas."""
import bench
import synth


def test_mmr_sizes():
    sc = synth.config_mmr()
    assert sc.n_voxels == 344 * 344 * 127 == 15_028_672
    bins_per_subset = sc.n_radial * sc.n_planes * (sc.n_views // sc.n_subsets)
    assert bins_per_subset == 344 * 837 == 287_928


def test_algorithmic_bytes_per_launch_at_mmr_scale():
    sc = synth.config_mmr()
    N, Mi, f32 = sc.n_voxels, 287_928, 4
    # k_forward (FWD_DATA): reads x; reads b, r, mult, y and the stored sigma is not counted
    # (recomputable from the chord); writes y and mult * dy of the subset
    forward = f32 * (N + 4 * Mi + 2 * Mi)
    # k_backward (BWD_UPDATE): reads mult * dy of the subset and x, z, T; writes x and z
    backward = f32 * (Mi + 3 * N + 2 * N)
    # k_prior (dTV): reads x, q (3 components), z, T, side image; writes x, q (3), z
    prior = f32 * ((1 + 3 + 1 + 1 + 1) * N + (1 + 3 + 1) * N)
    assert bench.kernel_bytes(sc, "forward") == forward == 67_024_960
    assert bench.kernel_bytes(sc, "backward") == backward == 301_725_152
    assert bench.kernel_bytes(sc, "prior") == prior == 721_376_256


def test_whole_job_rate_of_replicas():
    # 4 replicas of 5 epochs each, the slowest rank taking 0.5 s: 40 epochs/s for the job
    assert bench.aggregate_rate(5, 4, 0.5) == 40.0
    assert bench.max_over_ranks(0.25) == 0.25  # no process group: the value itself
