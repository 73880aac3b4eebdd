"""Static check of bench.py (no GPU): every name a function of bench.py reads
without binding it must exist at module level or among the builtins, so a
misspelled or missing variable fails here instead of in the middle of a GPU
run."""
import builtins
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _unbound_reads(table, module_names, out):
    for child in table.get_children():
        if child.get_type() == "function":
            for sym in child.get_symbols():
                if sym.is_referenced() and sym.is_global() and not sym.is_declared_global():
                    name = sym.get_name()
                    if name not in module_names and not hasattr(builtins, name):
                        out.append(f"{child.get_name()}: {name}")
        _unbound_reads(child, module_names, out)


@pytest.mark.parametrize("script", ["bench.py", "__graft_entry__.py"])
def test_every_name_read_is_bound(script):
    path = os.path.join(ROOT, script)
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    missing = []
    _unbound_reads(top, module_names, missing)
    assert not missing, f"names read but bound nowhere in {script}: {missing}"


def test_the_check_sees_an_unbound_name():
    src = "import os\ndef f(x):\n    y = x + 1\n    return y + traffic\n"
    top = symtable.symtable(src, "<t>", "exec")
    module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    missing = []
    _unbound_reads(top, module_names, missing)
    assert missing == ["f: traffic"]
