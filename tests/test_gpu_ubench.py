"""The integer issue-rate measurement (pbvd_measure_int_rate) behind the
roofline's denominator: every instruction kind reports a rate no higher than
the issue limit of 4 schedulers x 32 lanes per SM and clock, and mixing a
logic op with a multiply-add (two pipes) is not slower than either alone."""
import pytest

from paper_1608_00066_gb300 import pbvd

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def test_rates_within_the_issue_limit():
    rates = {name: pbvd.pbvd_measure_int_rate(op) for op, name in pbvd.INT_RATE_OPS.items()}
    for name, r in rates.items():
        assert 8.0 <= r <= 4 * 32 * 1.05, (name, r)
    assert rates["lop3+imad"] >= 0.95 * max(rates["lop3"], rates["imad"]), rates


def test_rejects_unknown_op():
    for op in (-1, 7):
        with pytest.raises(pbvd.PbvdError) as ei:
            pbvd.pbvd_measure_int_rate(op)
        assert ei.value.code == pbvd.PBVD_EINVAL
