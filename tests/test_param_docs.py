"""Every key bbc_set_param accepts is readable through bbc_get_param and
documented in the interface header, and the header documents no key the
library does not accept (a check on the sources, no GPU needed)."""

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _function_body(src, name):
    start = src.index(f"int {name}(")
    depth, i = 0, src.index("{", start)
    for j in range(i, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[i:j + 1]
    raise AssertionError(f"unterminated {name}")


def _keys(body):
    return set(re.findall(r'k == "([a-z_0-9]+)"', body))


def test_setter_getter_and_header_name_the_same_parameters():
    api = open(os.path.join(ROOT, "paper_2604_01960_gb300", "csrc", "api.cu")).read()
    hdr = open(os.path.join(ROOT, "include", "bbc.h")).read()
    set_keys = _keys(_function_body(api, "bbc_set_param"))
    get_keys = _keys(_function_body(api, "bbc_get_param"))
    assert len(set_keys) >= 20
    assert set_keys == get_keys
    # the header's parameter list: lines of the form ' *   "key"  description'
    documented = set(re.findall(r'^ \*\s+"([a-z_0-9]+)"\s', hdr, flags=re.M))
    assert set_keys <= documented, f"undocumented: {sorted(set_keys - documented)}"
    assert documented <= set_keys, f"documented but not accepted: {sorted(documented - set_keys)}"
