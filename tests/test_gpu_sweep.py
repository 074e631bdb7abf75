"""The table-scaling sweep's extremes on the GPU: a 5x10^7-sector master table (4.3 GB of slots,
far outside L2) checked at full table size against the plan's plant log, and a 10^3-sector table
planted at 10% density (every master cluster planted about 200 times) checked against the
oracle in full."""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def device_masters(file_nsect, mseed):
    mplan = synth.Plan(0, mseed, 0, file_nsect, np.zeros(0, np.int32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    base = mplan.file_base()
    base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
    masters = torch.empty(mplan.n_master_sectors * SECTOR, dtype=torch.uint8, device="cuda")
    mplan.masters_device(masters.data_ptr(), base_d.data_ptr())
    torch.cuda.synchronize()
    files = [(masters.data_ptr() + int(base[f]) * SECTOR, int(file_nsect[f]) * SECTOR) for f in range(file_nsect.size)]
    return masters, files


def device_image(plan):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    keep = [dev(plan.plant_file.view(np.uint8)), dev(plan.plant_fcluster.view(np.uint8)), dev(plan.plant_over),
            dev(plan.file_nsect.view(np.uint8)), dev(synth.vocab(plan.image_seed))]
    image = torch.empty(plan.n_bytes, dtype=torch.uint8, device="cuda")
    plan.image_device(image.data_ptr(), dev_plan=tuple(k.data_ptr() for k in keep))
    torch.cuda.synchronize()
    return image


def test_fifty_million_sector_table(cv):
    file_nsect, mseed = synth.sweep_master_set(50_000_000)
    masters, files = device_masters(file_nsect, mseed)
    with cv.master_build(files) as m:
        del masters
        info = m.info()
        assert info["n_kept"] == 50_000_000 and info["n_unique"] == 50_000_000
        assert info["n_slots"] == 1 << 27
        plan = synth.make_plan_density(31, 1 << 20, file_nsect, 0.1, mseed)
        image = device_image(plan)
        with cv.scan(m, [image]) as r:
            got = r.matches(0)
        exp = plan.expected_intact()
        assert exp.size > 90_000
        assert np.array_equal(got, exp)
        # spot-check planted sectors byte for byte against the generator's masters
        img = image.cpu().numpy().reshape(-1, SECTOR)
        for t in got[:: max(1, got.size // 50)]:
            ref = plan.master_host(int(t["file_id"]), int(t["file_sector"]), 1)
            assert np.array_equal(img[t["disk_sector"]], ref)


def test_small_table_dense_repeats_against_oracle(cv):
    file_nsect, mseed = synth.sweep_master_set(1000)
    plan = synth.make_plan_density(32, 131072, file_nsect, 0.1, mseed)
    img = plan.image_host()
    files = plan.masters_host()
    want = oracle.match_hash(img, files)
    assert want.size > 10_000  # about 10% of the 131,072 sectors, less the overwrites
    image = torch.from_numpy(img).cuda()
    for bloom in (0, cv.CV_BLOOM_AUTO):
        with cv.master_build(files, bloom_bits_per_key=bloom) as m:
            with cv.scan(m, [image]) as r:
                assert np.array_equal(r.matches(0), want), bloom
