"""The seeded input generator: determinism and the structure the workloads rely on."""
import numpy as np

from paper_2402_02273_gb300 import phantom


def test_splitmix_stream_is_fixed():
    # SplitMix64 of counter 0 with seed 0 / stream 0 is a fixed number on every machine
    a = phantom.uniform(0, 0, 4)
    b = phantom.uniform(0, 0, 4)
    assert np.array_equal(a, b)
    assert np.all((a >= 0) & (a < 1))
    assert not np.array_equal(a, phantom.uniform(1, 0, 4))
    assert not np.array_equal(a, phantom.uniform(0, 1, 4))
    big = phantom.uniform(3, 2, 200000)
    assert abs(big.mean() - 0.5) < 0.005 and abs(big.var() - 1 / 12) < 0.002


def test_head_phantom_structure():
    lab = phantom.head_labels((32, 32, 32), seed=0)
    counts = np.bincount(lab.ravel(), minlength=4)
    assert counts[phantom.LABEL_WHITE] > 0 and counts[phantom.LABEL_GRAY] > 0
    assert counts[phantom.LABEL_BACKGROUND] > 0 and counts[phantom.LABEL_CSF] > 0
    # corners are outside the head
    assert lab[0, 0, 0] == phantom.LABEL_BACKGROUND
    # the default seed site lies in white matter
    x, y, z = phantom.seed_centre((32, 32, 32))
    assert lab[int(round(z)), int(round(y)), int(round(x))] == phantom.LABEL_WHITE


def test_diffusion_field_values_are_fp32_exact_and_tissue_only():
    lab = phantom.head_labels((24, 20, 28), seed=5)
    D = phantom.diffusion_field(lab, seed=5, noise=0.1)
    assert np.array_equal(D, D.astype(np.float32).astype(np.float64))
    assert np.all(D[lab <= phantom.LABEL_CSF] == 0)
    white = D[lab == phantom.LABEL_WHITE]
    assert white.min() >= 0.13 * 0.9 * (1 - 1e-7) and white.max() <= 0.13 * 1.1 * (1 + 1e-7)
    clean = phantom.diffusion_field(lab, seed=5)
    assert set(np.unique(clean)) <= {0.0, np.float64(np.float32(0.013)), np.float64(np.float32(0.13))}


def test_case_is_reproducible():
    D1, u1 = phantom.case(16, seed=3, noise=0.1)
    D2, u2 = phantom.case(16, seed=3, noise=0.1)
    assert np.array_equal(D1, D2) and np.array_equal(u1, u2)
    assert u1.max() <= 0.8 and u1.max() > 0.5


def test_batch_case_ranges():
    for i in range(6):
        c = phantom.batch_case(i)
        assert c["n"] in (96, 112, 128, 144, 160)
        assert 0.01 <= c["rho"] <= 0.05 and 0.5 <= c["dscale"] <= 2.0
        assert c["D"].shape == (c["n"],) * 3 and c["u0"].max() > 0.5


def test_zero_row_count_helper_on_hand_cases():
    """The host count the GPU tests compare et_get_zero_rows with: a lone
    voxel with D > 0 has no face with D > 0 on both sides (conservative: every
    row is empty), but its literal row has 2 D_p towards -e and its +x / +y /
    +z neighbours' literal rows carry D_p + D_q towards it."""
    import numpy as np
    from zero_rows import zero_row_voxels
    D = np.zeros((3, 4, 40))
    assert zero_row_voxels(D, "conservative") == D.size
    assert zero_row_voxels(D, "literal") == D.size
    D[1, 2, 5] = 0.1
    assert zero_row_voxels(D, "conservative") == D.size
    # literal: rows of voxel (z1, y2, x5) and its -x / -y / -z neighbours are
    # not empty: three warp rows of 32 voxels (y2 and y1 of z1, y2 of z0)
    assert zero_row_voxels(D, "literal") == D.size - 3 * 32
    D[1, 2, 6] = 0.1  # a face with D > 0 on both sides
    assert zero_row_voxels(D, "conservative") == D.size - 32
