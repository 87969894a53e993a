import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """List the parity comparisons that needed the conditioning fallback or
    excused a hybrid-flag mismatch (see tests/parity_log.py)."""
    from tests import parity_log
    recs = parity_log.RECORDS
    if not recs:
        return
    path = os.environ.get("WENO_PARITY_LOG")
    if path:
        parity_log.dump(path)
    loose = [r for r in recs if r["level"] != "strict" or r["n_flag_mismatch"]]
    tr = terminalreporter
    tr.section("parity bars")
    levels = {k: sum(r["level"] == k for r in recs) for k in ("strict", "terms", "kappa")}
    tr.write_line(f"{len(recs)} comparisons: {levels['strict']} strict, {levels['terms']} on the flux-term "
                  f"scale, {levels['kappa']} on the oracle's sensitivity; "
                  f"{sum(bool(r['n_flag_mismatch']) for r in recs)} with excused flag mismatches")

    def f(x):
        return "-" if x is None else f"{x:.1e}"

    for r in loose:
        tr.write_line(f"  {r['test']} [{r['label']}]: {r['level']}, rel {f(r['rel_max'])}, "
                      f"rel to terms {f(r['rel_terms_max'])}, kappa {f(r['kappa_max'])}, bar {f(r['bar_max'])}, "
                      f"cap {f(r['cap'])}, flags {r['n_flag_mismatch']} "
                      f"(max |sigma/eps_h-1| {r['max_flag_window']:.1e})")
