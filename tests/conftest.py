import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle test that takes tens of seconds")
    config.addinivalue_line(
        "markers", "late: run after every other test, so that under -x a failure in one of them "
        "(tests of recently added paths) cannot keep the others from running")


def pytest_collection_modifyitems(session, config, items):
    # stable sort: established tests keep their order; late ones follow, by
    # the marker's optional rank (lowest first); the no-allocation entry
    # point's file comes after all of them
    def key(it):
        if it.fspath.basename == "test_zz_no_alloc.py":
            return (2, 0)
        mk = it.get_closest_marker("late")
        return (0, 0) if mk is None else (1, mk.args[0] if mk.args else 0)
    items.sort(key=key)
