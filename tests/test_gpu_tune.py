"""The autotuners: the kernel-configuration tuner leaves the bits unchanged,
and the batch geometry tuner's choice decodes exactly like the oracle run
with the chosen (D, L)."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth, tune

from gpu_util import mother_llr, oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def test_kernel_autotune_keeps_bits():
    spec = synth.K7_R12
    f = synth.make_frame(spec, 200000, 2.0, seed=31)
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    d = torch.from_numpy(f.llr).cuda()
    cfg, ms = dec.autotune(d, f.n_stages, reps=2)
    assert cfg["threads_per_pair"] in (1, 2, 4, 8, 16, 32) and ms > 0
    assert dec.get_config(f.n_stages)["threads_per_pair"] == cfg["threads_per_pair"]
    out = dec.decode(d, f.n_stages)
    torch.cuda.synchronize()
    got = np.unpackbits(out.cpu().numpy(), bitorder="little")[:f.n_stages]
    assert np.array_equal(got, oracle_bits(spec, f.llr, f.n_stages, 512, 42))


def test_batch_geometry_tuner_choice_matches_oracle():
    frames = synth.batch_frames(90, seed=4003)
    llrs = [torch.from_numpy(f.llr).cuda() for f in frames]
    outs = [torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda") for f in frames]
    choice, ms, trials = tune.tune_batch_geometry(frames, [x.data_ptr() for x in llrs],
                                                  [o.data_ptr() for o in outs], candidates=(512, 2048), reps=1)
    assert len(trials) == 2 ** len({f.spec.name for f in frames}) and ms > 0
    decs = {n: pbvd.Decoder(synth.CODES[n].K, synth.CODES[n].gens, synth.CODES[n].puncture, *choice[n])
            for n in choice}
    pbvd.pbvd_decode_batch(tune.make_items(frames, decs, [x.data_ptr() for x in llrs],
                                           [o.data_ptr() for o in outs]))
    torch.cuda.synchronize()
    for f, o in zip(frames, outs):
        D, L = choice[f.spec.name]
        want = oracle.viterbi_block(f.spec.K, f.spec.gens, mother_llr(f.spec, f.llr, f.n_stages), D, L)
        assert np.array_equal(np.unpackbits(o.cpu().numpy(), bitorder="little")[:f.n_stages], want)


def _auto_threads(N, pairs, sms):
    """The documented automatic rule of a device decode: the fewest threads
    per pair (a power of two) that give about 1.5 warps per SM scheduler,
    with at most 64 states per thread (32 above 64 states)."""
    tmin = 1
    while N // tmin > (32 if N > 64 else 64):
        tmin *= 2
    want = -(-(sms * 4 * 32 * 3 // 2) // pairs)
    T = 1
    while T < want and T < 32:
        T *= 2
    return min(max(T, tmin), 32, N // 2)


@pytest.mark.parametrize("spec,D", [(synth.K7_R12, 512), (synth.K7_R12, 256), (synth.K9_R13, 1024)])
def test_automatic_configuration_follows_the_documented_rule(spec, D):
    """pbvd_get_config reports the rule the header documents: at the
    2^24-bit stream's size two threads per pair in one-warp CTAs for the
    64-state code at D = 512, one at D = 256, eight for the 256-state code;
    shorter streams take more threads per pair."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    dec = pbvd.Decoder(spec.K, spec.gens, None, D, 42)
    for n in (1 << 24, 1 << 22, 1 << 20):
        pairs = -(-(-(-n // D)) // 2)
        cfg = dec.get_config(n)
        T = _auto_threads(1 << (spec.K - 1), pairs, sms)
        if pairs <= sms:
            continue  # few pairs: shared-memory survivors, CTA of one group
        assert cfg["threads_per_pair"] == T, (n, cfg, T)
        assert cfg["survivors_in_smem"] == 0
        assert cfg["cta_threads"] == (32 if T <= 2 else max(T, 64)), (n, cfg)
    dec.close()
