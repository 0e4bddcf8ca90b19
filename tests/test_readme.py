"""The usage the repository's front page shows stays valid: its Python block
compiles and every `api.` / `S.` name it uses (code and table) exists in the
package."""
import os
import re

from paper_1711_00289_gb300 import api
from paper_1711_00289_gb300 import soundings as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _readme():
    with open(os.path.join(ROOT, "README.md")) as f:
        return f.read()


def test_python_block_compiles():
    blocks = re.findall(r"```python\n(.*?)```", _readme(), re.S)
    assert blocks
    for b in blocks:
        compile(b, "README.md", "exec")


def test_names_exist():
    text = _readme()
    names = set(re.findall(r"\bapi\.([A-Za-z_]\w*)", text))
    assert {"deep_shallow", "PreparedStep", "HostPipeline", "ColumnModel"} <= names
    for n in names:
        assert hasattr(api, n), f"README names api.{n}"
    for n in set(re.findall(r"\bS\.([A-Za-z_]\w*)", text)):
        assert hasattr(S, n), f"README names soundings.{n}"
